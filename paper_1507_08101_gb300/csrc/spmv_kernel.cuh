// The augmented SELL-C-sigma SpMMV kernel (GHOST, Sec. "Kernel fusion"):
//
//     y = alpha (A - gamma I) x + beta y,  <y,y>, <x,y>, <x,x>,  z = delta z + eta y
//
// in one pass over the matrix.
//
// Mapping.  A block vector of width w (row-major, "interleaved", which the
// paper finds faster than column-major, Sec. "Block vectors") is padded to
// WP = next power of two <= 32.  Each lane owns CPL consecutive columns
// (a 16-byte vector of x when possible) and G = WP / CPL lanes share one row,
// so a warp covers R = 32 / G rows.  For w = 1 that is one row per lane: with
// C = 32 a warp reads 32 consecutive values and 32 consecutive column indices
// of a chunk column per step -- the coalescing the SELL layout was designed for
// (chunk entries stored column-wise).  For wider blocks the G lanes of a row
// read its x row as whole 16-byte vectors, so every gathered x row is one
// contiguous 8*w- or 4*w-byte line.
//
// Matrix values and indices are read once, with the streaming (evict-first)
// cache hint; x goes through the read-only path so that its reuse stays in L1
// and L2.  Each row runs only to its own length (the per-slot length), so
// padding is never read or multiplied.
//
// The grid is persistent (at most SMs x resident blocks) and walks the rows
// in a block-strided loop.  Dot products are reduced in a fixed order: lanes
// of a warp by xor shuffles, warps of a block through shared memory, blocks by
// the last block to finish (per-block partials + an atomic ticket), so the
// result is deterministic and no block ever waits for another.
#pragma once

#include <type_traits>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "common.cuh"

namespace sp {

constexpr int kSpmvThreads = 256;  // batched and sampled kernels
constexpr int kSpmvWarps = kSpmvThreads / 32;
// Block size of the main product kernel (warps per block, compile-time knob).
// Larger blocks put more of one SM's warps on adjacent partition ranges.
#ifndef SP_BLOCK_WARPS
#define SP_BLOCK_WARPS 32
#endif
constexpr int kMainWarps = SP_BLOCK_WARPS;
constexpr int kMainThreads = 32 * kMainWarps;
constexpr int kMaxTileW = 32;

struct SpmvArgs {
    const void *val;
    const int32_t *col;
    const int64_t *chunkptr;
    const int32_t *chunklen;  // null: the row loop runs per lane (see row_product_ls)
    const int32_t *slotlen;
    const int32_t *perm;  // null: identity (sigma = 1)
    int64_t nrows;
    int64_t nslots;
    int32_t C;
    int32_t w;
    const void *x;
    int64_t xrs, xcs;
    void *y;
    int64_t yrs, ycs;
    void *z;
    int64_t zrs, zcs;
    uint32_t flags;
    double alpha, beta, delta, eta;
    double *dot;
    int32_t dot_stride, dot_off;
    double *partials;
    unsigned *ticket;
    const int32_t *sched;    // moving-front schedule of this grid (null: see wbounds)
    int32_t sched_rounds;
    const int32_t *wbounds;  // static partition of this grid (null: block-strided loop)
    int32_t nsm;             // SMs the grid was sized for
    int32_t log2_tpr;        // threads per row T = 2^log2_tpr (lanes splitting one row's entries)
    int32_t log2C;           // log2 of C when C is a power of two, else -1
    int32_t dyn_grab;        // > 0: warps take runs of this many slots from a counter (no dots)
    const Pattern *wbounds_src;  // host side only: where the launcher finds the partition
    // C = V^T y formed with the product (kernels with MV > 0): V is nrows x
    // vty_m (row-major, leading dimension vty_ldv), C is vty_m x w (vty_ldc)
    const double *vty_V;
    int64_t vty_ldv;
    int32_t vty_m;
    int32_t vty_vec2;  // rows of V start on 16 bytes: V read as pairs of doubles
    double *vty_C;
    int64_t vty_ldc;
    double gamma[kMaxTileW];
};

// Tuning knobs (compile-time): unroll depth of the row loop for narrow lanes,
// and the minimum resident blocks per SM requested for the width-1 variants.
#ifndef SP_UNROLL_NARROW
#define SP_UNROLL_NARROW 8
#endif
#ifndef SP_UNROLL_WIDE
#define SP_UNROLL_WIDE 2
#endif
#ifndef SP_UNROLL_WIDE_F32
#define SP_UNROLL_WIDE_F32 4
#endif
#ifndef SP_MINB_W1
#define SP_MINB_W1 1
#endif
// minimum resident blocks per SM requested for wide blocks (WP >= 8):
// measured best at 3 (float64 vectors) and 4 (float32 vectors)
#ifndef SP_MINB_WIDE_F64
#define SP_MINB_WIDE_F64 3
#endif
#ifndef SP_MINB_WIDE_F32
#define SP_MINB_WIDE_F32 4
#endif

template <class VT, class XT>
struct AccOf { using T = float; };
template <>
struct AccOf<double, double> { using T = double; };

// Widest run of columns one lane owns (compile-time knob per vector precision).
#ifndef SP_CPL_MAX_F64
#define SP_CPL_MAX_F64 4
#endif
#ifndef SP_CPL_MAX_F32
#define SP_CPL_MAX_F32 8
#endif

template <class XT, int WP>
__host__ __device__ constexpr int cols_per_lane() {
    return (sizeof(XT) == 8 ? SP_CPL_MAX_F64 : SP_CPL_MAX_F32) < WP ? (sizeof(XT) == 8 ? SP_CPL_MAX_F64 : SP_CPL_MAX_F32)
                                                                      : WP;
}

// Host mirror of cols_per_lane for a runtime width.
inline int host_cols_per_lane(size_t xsize, int w) {
    int wp = 1;
    while (wp < w) wp <<= 1;
    int c = xsize == 8 ? SP_CPL_MAX_F64 : SP_CPL_MAX_F32;
    return c < wp ? c : wp;
}

// Threads per row.  A chunk of C rows is read by C*T lanes when
// C * T * G = 32: lane (r, t) takes the entries j = t, t + T, t + 2T, ... of
// row r, so for each step the warp's value and index loads are one
// contiguous run of 32 entries (T rows' worth of chunk columns); long rows
// get T lanes each.  For C >= 32 / G (or C not a power of two) T = 1.
inline int host_log2_tpr(int C, int G) {
    int rows_t1 = 32 / G;
    if (C >= rows_t1 || (C & (C - 1)) != 0) return 0;
    int t = rows_t1 / C, l = 0;
    while ((1 << l) < t) ++l;
    return l;
}

template <class AT, class VT>
__device__ __forceinline__ AT val_to_acc(VT v) { return (AT)v; }
template <>
__device__ __forceinline__ float val_to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// Precision changes between float64 vectors and float32 row sums, written with
// integer instructions: on GB300 a float64 <-> float32 conversion instruction
// runs on the float64 pipe, which issues about two lanes per SM and cycle, so
// one conversion per gathered x element (values in float32 or bfloat16 with
// float64 vectors) would cost as much as the float64 product it replaces.
//
// narrow_fast: float64 -> float32, round to nearest even, bit-identical to the
// conversion instruction whenever the result is a normal float or a rounded
// zero (|d| < 2^-150); every other input (results in the float32 subnormal
// range, overflow, infinities, NaN) sets `bad`, and the caller recomputes
// with the conversion instruction (x_to_acc<..., true>).
__device__ __forceinline__ float narrow_fast(double d, int &bad) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned s = hi & 0x80000000u;
    const unsigned e = (hi >> 20) & 0x7ffu;
    // exponent rebiased by 1023 - 127 = 896 (no borrow for e >= 897), 20 + 3
    // mantissa bits from hi, 3 from lo; then round on the 29 dropped bits
    unsigned f = s | (((hi - 0x38000000u) << 3) & 0x7ffffff8u) | (lo >> 29);
    const unsigned r = lo & 0x1fffffffu;
    f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
    const bool tiny = e <= 872u;                  // |d| < 2^-150 (or zero): rounds to a signed zero
    const bool normal = e - 897u <= 253u;         // result exponent 1..254 before rounding
    bad |= (tiny || normal) ? 0 : 1;
    return __uint_as_float(tiny ? s : f);
}

// widen_bits: float32 -> float64 (exact) for every input, by integer
// instructions (normal, zero, subnormal, infinity, NaN with its payload).
__device__ __forceinline__ double widen_bits(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned s = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned hi = s | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0u) {
        // zero, or a subnormal m 2^-149: the leading one moves to bit 23
        const int sh = __clz(m) - 8;
        const unsigned mm = (m << (sh & 31)) & 0x7fffffu;
        hi = m == 0u ? s : (s | ((unsigned)(897 - sh) << 20) | (mm >> 3));
        lo = m == 0u ? 0u : (mm << 29);
    }
    if (e == 255u) hi = s | 0x7ff00000u | (m >> 3);
    return __hiloint2double((int)hi, (int)lo);
}

// A gathered x element in the accumulation precision.  EXACT: the conversion
// instruction (the recompute path of narrow_fast's rare inputs).
template <class AT, class XT, bool EXACT>
__device__ __forceinline__ AT x_to_acc(XT v, int &bad) {
    if constexpr (std::is_same<AT, float>::value && std::is_same<XT, double>::value && !EXACT)
        return narrow_fast(v, bad);
    else
        return (AT)v;
}

// A row sum in the vector precision.
template <class XT, class AT>
__device__ __forceinline__ XT acc_to_x(AT v) {
    if constexpr (std::is_same<AT, float>::value && std::is_same<XT, double>::value)
        return widen_bits(v);
    else
        return (XT)v;
}

// Loads of the matrix stream (values, column indices): read once, so they
// should not displace x from the caches.  SP_STREAM_NOALLOC selects the
// read-only path without L1 allocation; otherwise the evict-first hint.
#ifndef SP_STREAM_NOALLOC
#define SP_STREAM_NOALLOC 0
#endif
#if SP_STREAM_NOALLOC
__device__ __forceinline__ double ld_stream(const double *p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ __nv_bfloat16 ld_stream(const __nv_bfloat16 *p) {
    unsigned short v;
    asm("ld.global.nc.L1::no_allocate.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return __ushort_as_bfloat16(v);
}
#else
template <class T>
__device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
#endif
// The matrix stream: evict-first (ST) where every sector a step touches is
// read whole by that step, else a normal load so that a sector read in parts
// by consecutive steps stays cached between them.
template <bool ST, class T>
__device__ __forceinline__ T ld_mat(const T *p) {
    if constexpr (ST) return ld_stream(p);
    else return __ldg(p);
}

// Epilogue arithmetic written as explicit fused multiply-adds and rounded
// products (never left to the compiler's contraction), so that each kernel
// that applies the same epilogue to the same row sum gets the same bits, with
// as few float64 instructions as the formula allows (GB300's float64 rate is
// low enough to bound these kernels):
//   y = alpha * fma(-gamma, x_i, t);  y = fma(beta, y_old, y)
//   z = fma(eta, y, delta * z);       <.,.> accumulated with fma
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Load CPL consecutive columns of one row of a block vector.
// VEC: all CPL columns valid, unit column stride, address aligned to
// min(16, CPL*sizeof(XT)) bytes.
template <class XT, int CPL, bool VEC>
__device__ __forceinline__ void load_cols(const XT *__restrict__ p, int64_t cs, int nvalid, XT (&o)[CPL]) {
    if constexpr (VEC) {
        constexpr int B = CPL * (int)sizeof(XT);
        if constexpr (B % 16 == 0) {
#pragma unroll
            for (int q = 0; q < B / 16; ++q) {
                uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + q);
                memcpy(&o[q * (16 / sizeof(XT))], &u, 16);
            }
        } else if constexpr (B == 8) {
            uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
            memcpy(&o[0], &u, 8);
        } else {
            o[0] = __ldg(p);
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c) o[c] = c < nvalid ? __ldg(p + c * cs) : XT(0);
    }
}

// Plain (coherent) load/store of an output row: y and z are read and written.
template <class XT, int CPL, bool VEC>
__device__ __forceinline__ void load_out(const XT *p, int64_t cs, int nvalid, XT (&o)[CPL]) {
    if constexpr (VEC) {
        constexpr int B = CPL * (int)sizeof(XT);
        if constexpr (B % 16 == 0) {
#pragma unroll
            for (int q = 0; q < B / 16; ++q) {
                uint4 u = reinterpret_cast<const uint4 *>(p)[q];
                memcpy(&o[q * (16 / sizeof(XT))], &u, 16);
            }
        } else if constexpr (B == 8) {
            uint2 u = *reinterpret_cast<const uint2 *>(p);
            memcpy(&o[0], &u, 8);
        } else {
            o[0] = *p;
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c) o[c] = c < nvalid ? p[c * cs] : XT(0);
    }
}

// CS: store with the streaming hint (evict-first), for an output the call
// does not read again, so that written rows do not push x out of L2 (plain
// float64 product, Laplacian 256^3: 328 -> 314 us); SP_STORE_CS forces it on
// for every output (a knob)
#ifndef SP_STORE_CS
#define SP_STORE_CS 0
#endif
#ifndef SP_STORE_CS_PLAIN
#define SP_STORE_CS_PLAIN 1
#endif
template <bool CS, class T>
__device__ __forceinline__ void st_out(T *p, T v) {
    if constexpr (CS || SP_STORE_CS != 0) __stcs(p, v);
    else *p = v;
}
template <class XT, int CPL, bool VEC, bool CS = false>
__device__ __forceinline__ void store_out(XT *p, int64_t cs, int nvalid, const XT (&o)[CPL]) {
    if constexpr (VEC) {
        constexpr int B = CPL * (int)sizeof(XT);
        if constexpr (B % 16 == 0) {
#pragma unroll
            for (int q = 0; q < B / 16; ++q) {
                uint4 u;
                memcpy(&u, &o[q * (16 / sizeof(XT))], 16);
                st_out<CS>(reinterpret_cast<uint4 *>(p) + q, u);
            }
        } else if constexpr (B == 8) {
            uint2 u;
            memcpy(&u, &o[0], 8);
            st_out<CS>(reinterpret_cast<uint2 *>(p), u);
        } else {
            st_out<CS>(p, o[0]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (c < nvalid) st_out<CS>(p + c * cs, o[c]);
    }
}

// The last (fewer than U) entries of a row loop.  `steps` (1..U) is how
// many multiply-adds the warp has to issue: in the lockstep loop the entries
// left in the longest row of the chunk (the same for every lane of it), in
// the per-lane loop U.  Slot k of the unrolled
// sequence holds entry k - (U - steps), so the loads and gathers all go out
// at once, and a jump into the sequence (fall-through switch) issues exactly
// `steps` multiply-adds, in entry order: a multiply-add under a false
// predicate would cost as much as a real one on GB300's float64 pipe (a
// predicated-off lane still occupies its slot of the warp instruction).
template <class VT, class XT, class AT, int CPL, bool VEC, int U, bool EXACT, bool ST = true>
__device__ __forceinline__ void tail_steps(const VT *__restrict__ vp, const int32_t *__restrict__ cp, int C,
                                           int rest, int steps, const XT *__restrict__ xk, int64_t xrs,
                                           int64_t xcs, int nvalid, AT (&acc)[CPL], int &bad) {
    static_assert(U >= 1 && U <= 8, "tail unroll");
    const int sh = U - steps;
    int32_t cc[U];
    VT vv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const int e = k - sh;
        const bool ok = e >= 0 && e < rest;
        cc[k] = ok ? ld_mat<ST>(cp + (int64_t)e * C) : 0;
        vv[k] = ok ? ld_mat<ST>(vp + (int64_t)e * C) : VT(0);
    }
    if (nvalid <= 0) return;
    XT xv[U][CPL];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const int e = k - sh;
        if (e >= 0 && e < rest) {
            load_cols<XT, CPL, VEC>(xk + (int64_t)cc[k] * xrs, xcs, nvalid, xv[k]);
        } else {
#pragma unroll
            for (int c = 0; c < CPL; ++c) xv[k][c] = XT(0);
        }
    }
    auto step = [&](int k) {
        if (k - sh < rest) {
            const AT v = val_to_acc<AT, VT>(vv[k]);
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] = fma(v, x_to_acc<AT, XT, EXACT>(xv[k][c], bad), acc[c]);
        }
    };
    switch (sh) {
        case 0: if (U > 0) step(0); [[fallthrough]];
        case 1: if (U > 1) step(1); [[fallthrough]];
        case 2: if (U > 2) step(2); [[fallthrough]];
        case 3: if (U > 3) step(3); [[fallthrough]];
        case 4: if (U > 4) step(4); [[fallthrough]];
        case 5: if (U > 5) step(5); [[fallthrough]];
        case 6: if (U > 6) step(6); [[fallthrough]];
        case 7: if (U > 7) step(7); [[fallthrough]];
        default: break;
    }
}

// Lockstep form of row_product: every lane of a chunk steps through the
// chunk's length clen (the same for all of them), and the entries past a lane's
// own row length are predicated off.  The warp then issues one step per column
// of the chunk instead of running the lanes' different tails one after the
// other (on the float64 pipe a step costs the same whatever lanes are active).
// The products are added in the order j = 0, 1, ..., len - 1, as in
// row_product, so the two give identical sums.
// SP_LOCKSTEP: 0 never, 1 where it pays (float64 products: always for block
// vectors, for single vectors when the row lengths inside a warp's slots
// spread widely), 2 always.
#ifndef SP_LOCKSTEP
#define SP_LOCKSTEP 1
#endif

// Longest run of row iterations over which a lane of a float32-vector product
// accumulates its dot products in float (SP_DOT_RUN_F32, defined in the header).
static_assert(SP_DOT_RUN_F32 >= 1, "dot run length");
#ifndef SP_LS_SPREAD
#define SP_LS_SPREAD 0.3
#endif
#ifndef SP_LS_SPREAD_DOTS
#define SP_LS_SPREAD_DOTS 0.15
#endif
template <class VT, class XT, class AT, int CPL, bool VEC, int U, bool EXACT = false, bool ST = true>
__device__ __forceinline__ void row_product_ls(const VT *__restrict__ vp, const int32_t *__restrict__ cp, int C,
                                               int len, int clen, const XT *__restrict__ xk, int64_t xrs,
                                               int64_t xcs, int nvalid, AT (&acc)[CPL], int &bad) {
    int j = 0;
    for (; j + U <= clen; j += U) {
        int32_t cc[U];
        VT vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = j + u < len;
            cc[u] = ok ? ld_mat<ST>(cp + (int64_t)u * C) : 0;
            vv[u] = ok ? ld_mat<ST>(vp + (int64_t)u * C) : VT(0);
        }
        vp += (int64_t)U * C;
        cp += (int64_t)U * C;
        if (nvalid > 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j + u < len) {
                    XT xv[CPL];
                    load_cols<XT, CPL, VEC>(xk + (int64_t)cc[u] * xrs, xcs, nvalid, xv);
                    AT v = val_to_acc<AT, VT>(vv[u]);
#pragma unroll
                    for (int c = 0; c < CPL; ++c) acc[c] = fma(v, x_to_acc<AT, XT, EXACT>(xv[c], bad), acc[c]);
                }
            }
        }
    }
    if (clen > j)
        tail_steps<VT, XT, AT, CPL, VEC, U, EXACT, ST>(vp, cp, C, len - j, clen - j, xk, xrs, xcs, nvalid, acc, bad);
}

// Row sums t[c] = sum_j val(s,j) * x[col(s,j), k0 + c] for the row in one slot.
// U value/index loads and U gathers are in flight per step; the last
// (len mod U) entries are issued the same way under a predicate, so a short
// row (fewer than U entries) costs one round trip, not one per entry.  The
// products are added in the order j = 0, 1, ..., len - 1 in every case.
template <class VT, class XT, class AT, int CPL, bool VEC, int U, bool EXACT = false, bool ST = true>
__device__ __forceinline__ void row_product(const VT *__restrict__ vp, const int32_t *__restrict__ cp, int C,
                                            int len, const XT *__restrict__ xk, int64_t xrs, int64_t xcs,
                                            int nvalid, AT (&acc)[CPL], int &bad) {
    int j = 0;
    for (; j + U <= len; j += U) {
        int32_t cc[U];
        VT vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = ld_mat<ST>(cp + (int64_t)u * C);
            vv[u] = ld_mat<ST>(vp + (int64_t)u * C);
        }
        vp += (int64_t)U * C;
        cp += (int64_t)U * C;
        if (nvalid > 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                XT xv[CPL];
                load_cols<XT, CPL, VEC>(xk + (int64_t)cc[u] * xrs, xcs, nvalid, xv);
                AT v = val_to_acc<AT, VT>(vv[u]);
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = fma(v, x_to_acc<AT, XT, EXACT>(xv[c], bad), acc[c]);
            }
        }
    }
    // lanes run rows of their own lengths here, so no count shorter than U
    // bounds every lane's tail: all U steps, each under its lane's predicate
    const int rest = len - j;
    if (rest > 0) tail_steps<VT, XT, AT, CPL, VEC, U, EXACT, ST>(vp, cp, C, rest, U, xk, xrs, xcs, nvalid, acc, bad);
}

// row_product with the index and value loads one batch ahead: batch b + 1's
// U loads go out before batch b's gathers are consumed, so a row of n
// batches costs about n + 1 memory round trips instead of 2n.  Every load and
// multiply-add is under its lane's predicate (j + u < len), which on the
// float32 pipe costs little; the products are added in the order
// j = 0, 1, ..., len - 1, so the sums equal row_product's bit for bit.
template <class VT, class XT, class AT, int CPL, bool VEC, int U, bool EXACT = false, bool ST = true>
__device__ __forceinline__ void row_product_pipe(const VT *__restrict__ vp, const int32_t *__restrict__ cp, int C,
                                                 int len, const XT *__restrict__ xk, int64_t xrs, int64_t xcs,
                                                 int nvalid, AT (&acc)[CPL], int &bad) {
    int32_t cc[U];
    VT vv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const bool ok = u < len;
        cc[u] = ok ? ld_mat<ST>(cp + (int64_t)u * C) : 0;
        vv[u] = ok ? ld_mat<ST>(vp + (int64_t)u * C) : VT(0);
    }
    for (int j = 0; j < len; j += U) {
        int32_t cn[U];
        VT vn[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = j + U + u < len;
            cn[u] = ok ? ld_mat<ST>(cp + (int64_t)(j + U + u) * C) : 0;
            vn[u] = ok ? ld_mat<ST>(vp + (int64_t)(j + U + u) * C) : VT(0);
        }
        if (nvalid > 0) {
            XT xv[U][CPL];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j + u < len) {
                    load_cols<XT, CPL, VEC>(xk + (int64_t)cc[u] * xrs, xcs, nvalid, xv[u]);
                } else {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) xv[u][c] = XT(0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j + u < len) {
                    const AT v = val_to_acc<AT, VT>(vv[u]);
#pragma unroll
                    for (int c = 0; c < CPL; ++c) acc[c] = fma(v, x_to_acc<AT, XT, EXACT>(xv[u][c], bad), acc[c]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = cn[u];
            vv[u] = vn[u];
        }
    }
}

// Per-warp float64 sums of the dot products in shared memory: the warp's
// running bank while it works (float32 vectors, see k_spmmv), then the input of
// the block-level reduction.
__device__ __forceinline__ double (*dot_smem())[3][kMaxTileW] {
    __shared__ double sred[kMainWarps][3][kMaxTileW];
    return sred;
}

// Final step of the fused reductions: per-block partial sums, and the last
// block to arrive adds them up in block order.  BANKED: the warp's sums so far
// are already in its row of dot_smem() and this call adds to them.
template <int CPL, int G, int DM, bool BANKED>
__device__ __forceinline__ void reduce_dots(const SpmvArgs &a, int k0, double (&dyy)[CPL], double (&dxy)[CPL],
                                            double (&dxx)[CPL]) {
    double (*sred)[3][kMaxTileW] = dot_smem();
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            if constexpr ((DM & 1) != 0) dyy[c] += __shfl_xor_sync(0xffffffffu, dyy[c], o);
            if constexpr ((DM & 2) != 0) dxy[c] += __shfl_xor_sync(0xffffffffu, dxy[c], o);
            if constexpr ((DM & 4) != 0) dxx[c] += __shfl_xor_sync(0xffffffffu, dxx[c], o);
        }
    }
    if (lane < G) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            int k = k0 + c;
            if (k < a.w) {
                if constexpr (BANKED) {
                    sred[warp][0][k] += dyy[c];
                    sred[warp][1][k] += dxy[c];
                    sred[warp][2][k] += dxx[c];
                } else {
                    sred[warp][0][k] = dyy[c];
                    sred[warp][1][k] = dxy[c];
                    sred[warp][2][k] = dxx[c];
                }
            }
        }
    }
    __syncthreads();
    const int nv = 3 * a.w;
    const int nb = gridDim.x;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        int q = t / a.w, k = t - q * a.w;
        double s = 0.0;
#pragma unroll
        for (int wi = 0; wi < kMainWarps; ++wi) s += sred[wi][q][k];
        a.partials[(int64_t)t * nb + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(a.ticket, 1u) == (unsigned)nb - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int t = warp; t < nv; t += kMainWarps) {
        int q = t / a.w, k = t - q * a.w;
        if (!(a.flags & (SP_SPMV_DOT_YY << q))) continue;
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(a.partials + (int64_t)t * nb + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.dot[(int64_t)q * a.dot_stride + a.dot_off + k] = s;
    }
    if (threadIdx.x == 0) *a.ticket = 0u;
}

// C = V^T y from the lanes' partial sums, in a fixed order like reduce_dots:
// lanes of a column group by an xor tree, the warps of a block in order, the
// blocks in order by the last block to arrive.  Value (p, k) is number
// p w + k (at most 8 x 8 of the 3 x 32 slots per warp and per block).
template <int CPL, int G, int MV>
__device__ __forceinline__ void reduce_vty(const SpmvArgs &a, int k0, double (&v)[MV][CPL]) {
    double (*sred)[3][kMaxTileW] = dot_smem();
    __shared__ int is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *mine = &sred[warp][0][0];
#pragma unroll
    for (int p = 0; p < MV; ++p)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
#pragma unroll
            for (int o = G; o < 32; o <<= 1) v[p][c] += __shfl_xor_sync(0xffffffffu, v[p][c], o);
            if (lane < G && p < a.vty_m && k0 + c < a.w) mine[p * a.w + k0 + c] = v[p][c];
        }
    __syncthreads();
    const int nv = a.vty_m * a.w;
    const int nb = gridDim.x;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int wi = 0; wi < kMainWarps; ++wi) s += (&sred[wi][0][0])[t];
        a.partials[(int64_t)t * nb + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(a.ticket, 1u) == (unsigned)nb - 1u);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int t = warp; t < nv; t += kMainWarps) {
        const int p = t / a.w, k = t - p * a.w;
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(a.partials + (int64_t)t * nb + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.vty_C[(int64_t)p * a.vty_ldc + k] = s;
    }
    if (threadIdx.x == 0) *a.ticket = 0u;
}

// Swizzle of the block index before it picks its slice of the partition: with
// SP_SWIZZLE blocks b, b + SMs, b + 2 SMs, ... (the blocks a one-wave launch
// usually places on one SM) own consecutive slices, so each SM works on one
// contiguous region and its L1 sees the x reuse of that region.
#ifndef SP_SWIZZLE
#define SP_SWIZZLE 0
#endif
// Latency overlap in the slot loop: issue the epilogue's loads before the row
// loop, and load the next slot's metadata while the current slot runs.
// Per vector precision: the float64 kernels are register bound, and the
// epilogue's early loads and the next slot's metadata cost them more than they
// hide (bench workload +4 %, Laplacian 256^3 +6 % without); the float32
// kernels gain from both.
#ifndef SP_EARLY_EPI_F64
#define SP_EARLY_EPI_F64 0
#endif
#ifndef SP_EARLY_EPI_F32
#define SP_EARLY_EPI_F32 1
#endif
// V^T y: rows of V read as pairs of doubles where they are 16-byte aligned (knob)
#ifndef SP_VTY_VEC2
#define SP_VTY_VEC2 1
#endif
// float-accumulated products: row loop with loads one batch ahead (knob)
#ifndef SP_PIPE_F32
#define SP_PIPE_F32 1
#endif
#ifndef SP_PREFETCH_META_F64
#define SP_PREFETCH_META_F64 0
#endif
#ifndef SP_PREFETCH_META_F32
#define SP_PREFETCH_META_F32 1
#endif
#ifndef SP_PREFETCH_META_F64_PLAIN
#define SP_PREFETCH_META_F64_PLAIN 0
#endif

// MT: rows may be split over T > 1 lanes (threads per row).  With MT false the
// kernel is compiled for T = 1 and carries none of the split-row logic.
// DM: the dot products compiled in (bit 0 <y,y>, bit 1 <x,y>, bit 2 <x,x>);
// the launcher uses 0, 3 (the pair of the bench product and of the KPM steps)
// or 7, and the flags pick which of them are written.
// EPI: the epilogue's arithmetic, fixed at compile time where the float64
// pipe binds (float64 vectors): 0 y = t; 1 y = alpha t + beta y (the
// Chebyshev step); 2 every augmentation by its runtime flag; 3 shift, scale
// and beta = 1 (dots and chain by their flags): y = alpha t - alpha gamma x_i
// + y_old in two fused multiply-adds.  A runtime
// flag that is off still costs: the compiler turns a short conditional into
// an unconditional operation and a select, and for float64 vectors that
// operation occupies the float64 pipe (Laplacian 256^3: three of every eleven
// float64 instructions per row were such).
template <class VT, class XT, int WP, bool VEC, int DM, bool MT, bool LS, int EPI, int MV = 0>
__global__ void __launch_bounds__(kMainThreads, kMainWarps > 8 ? 1 : (WP == 1 ? SP_MINB_W1 : WP < 8 ? 1 : sizeof(XT) == 8 ? SP_MINB_WIDE_F64 : SP_MINB_WIDE_F32))
    k_spmmv(const __grid_constant__ SpmvArgs a) {
    using AT = typename AccOf<VT, XT>::T;
    // dot accumulators per lane: float64 for float64 vectors; for float32
    // vectors float per lane over at most SP_DOT_RUN_F32 row iterations of the
    // warp, then a float xor tree across the lanes of each column and a float64
    // add into the warp's bank in shared memory (dot_flush), so the kernel
    // spends no float64 instruction per row and every term passes through at
    // most SP_DOT_RUN_F32 + 5 float additions
    using DT = typename std::conditional<sizeof(XT) == 8, double, float>::type;
    constexpr bool DOTS = DM != 0;
    constexpr bool BANK = DOTS && sizeof(XT) == 4;
    constexpr int CPL = cols_per_lane<XT, WP>();
    constexpr int G = WP / CPL;
    constexpr int R = 32 / G;
    constexpr int U = CPL >= 4 ? (sizeof(XT) == 4 ? SP_UNROLL_WIDE_F32 : SP_UNROLL_WIDE) : SP_UNROLL_NARROW / CPL;
    constexpr bool early_epi = sizeof(XT) == 8 ? SP_EARLY_EPI_F64 != 0 : SP_EARLY_EPI_F32 != 0;
    // the plain float64 product (no epilogue loads, no dots) has registers to
    // spare for the next slot's metadata
    constexpr bool prefetch_meta = sizeof(XT) == 8 ? (EPI == 0 ? SP_PREFETCH_META_F64_PLAIN != 0
                                                               : SP_PREFETCH_META_F64 != 0)
                                                   : SP_PREFETCH_META_F32 != 0;

    // evict-first matrix loads only where one warp step reads whole 32-byte
    // sectors of values and indices (the step covers R rows of a chunk column)
    constexpr bool ST = R * sizeof(int32_t) >= 32 && R * sizeof(VT) >= 32;
    // float accumulation: the row loop with its index and value loads one batch
    // ahead (measured faster for every pair but bfloat16 values with float32
    // vectors, which keeps the plain loop)
    constexpr bool pipe = std::is_same<AT, float>::value && SP_PIPE_F32 != 0 &&
                          !(std::is_same<VT, __nv_bfloat16>::value && std::is_same<XT, float>::value);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lt = MT ? a.log2_tpr : 0;     // T = 1 << lt lanes per row (runtime)
    const int T = 1 << lt;
    const int gl = lane % G;
    const int tt = (lane / G) & (T - 1);    // this lane's share of the row's entries
    const int rw = (lane / G) >> lt;        // row of the warp
    const int Rr = R >> lt;                 // rows per warp
    const unsigned rowmask = (G * T == 32) ? 0xffffffffu : (((1u << (G * T)) - 1u) << (rw * G * T));
    const int k0 = gl * CPL;
    const int nvalid = a.w - k0 < CPL ? a.w - k0 : CPL;
    const uint32_t f = a.flags;
    static_assert(EPI >= 2 || DM == 0, "compile-time epilogues 0 and 1 have no dots");
    static_assert(MV == 0 || (DM == 0 && !MT && std::is_same<XT, double>::value),
                  "V^T y: float64 vectors, no fused dots, one lane group per row");
    const bool shift = EPI == 3 || (EPI == 2 && (f & (SP_SPMV_SHIFT | SP_SPMV_VSHIFT)) != 0);
    const bool do_scale = EPI == 2 ? (f & SP_SPMV_SCALE) != 0 : EPI != 0;
    const bool do_axpby = EPI == 2 ? (f & SP_SPMV_AXPBY) != 0 : EPI != 0;
    const bool do_chain = EPI >= 2 && (f & SP_SPMV_CHAIN_AXPBY) != 0;
    const bool need_xi = shift || (DM != 0 && (f & (SP_SPMV_DOT_XY | SP_SPMV_DOT_XX)));
    const VT *__restrict__ val = (const VT *)a.val;
    const XT *__restrict__ x = (const XT *)a.x;
    XT *y = (XT *)a.y;
    XT *z = (XT *)a.z;
    const XT alpha = (XT)a.alpha, beta = (XT)a.beta, delta = (XT)a.delta, eta = (XT)a.eta;
    XT gam[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) gam[c] = (shift && k0 + c < a.w) ? (XT)a.gamma[k0 + c] : XT(0);

    DT dyy[(DM & 1) ? CPL : 1], dxy[(DM & 2) ? CPL : 1], dxx[(DM & 4) ? CPL : 1];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        if constexpr ((DM & 1) != 0) dyy[c] = DT(0);
        if constexpr ((DM & 2) != 0) dxy[c] = DT(0);
        if constexpr ((DM & 4) != 0) dxx[c] = DT(0);
    }

    // this lane's share of C = V^T y: V[i, p] y[i, k0 + c] summed over its rows
    double vacc[MV > 0 ? MV : 1][MV > 0 ? CPL : 1];
#pragma unroll
    for (int p = 0; p < (MV > 0 ? MV : 1); ++p)
#pragma unroll
        for (int c = 0; c < (MV > 0 ? CPL : 1); ++c) vacc[p][c] = 0.0;

    const XT *__restrict__ xk = x + (int64_t)k0 * a.xcs;

    if constexpr (BANK) {
        double (*bank)[3][kMaxTileW] = dot_smem();
        for (int t = lane; t < 3 * kMaxTileW; t += 32) bank[warp][t / kMaxTileW][t % kMaxTileW] = 0.0;
        __syncwarp();
    }
    // Called by every lane of the warp at the same points (once per uniform
    // iteration of the slot loops): after SP_DOT_RUN_F32 iterations the float
    // sums move into the warp's float64 bank.
    int dot_iters = 0;
    auto dot_tick = [&]() {
        if constexpr (BANK) {
            if (++dot_iters < SP_DOT_RUN_F32) return;
            dot_iters = 0;
            double (*bank)[3][kMaxTileW] = dot_smem();
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
#pragma unroll
                for (int o = G; o < 32; o <<= 1) {
                    if constexpr ((DM & 1) != 0) dyy[c] += __shfl_xor_sync(0xffffffffu, dyy[c], o);
                    if constexpr ((DM & 2) != 0) dxy[c] += __shfl_xor_sync(0xffffffffu, dxy[c], o);
                    if constexpr ((DM & 4) != 0) dxx[c] += __shfl_xor_sync(0xffffffffu, dxx[c], o);
                }
                if (lane < G && k0 + c < a.w) {
                    if constexpr ((DM & 1) != 0) bank[warp][0][k0 + c] += (double)dyy[c];
                    if constexpr ((DM & 2) != 0) bank[warp][1][k0 + c] += (double)dxy[c];
                    if constexpr ((DM & 4) != 0) bank[warp][2][k0 + c] += (double)dxx[c];
                }
                if constexpr ((DM & 1) != 0) dyy[c] = DT(0);
                if constexpr ((DM & 2) != 0) dxy[c] = DT(0);
                if constexpr ((DM & 4) != 0) dxx[c] = DT(0);
            }
        }
    };

    // one row slot: row sums, then y = alpha (t - gamma x_i) + beta y_i, dots, chain
    // Where a slot's row lives: its original row i (-1 for a padding row),
    // the offset of its first entry and its length.  Three independent loads.
    struct Meta {
        int64_t i, off;
        int len, clen;
    };
    auto meta_of = [&](int64_t s) {
        Meta m;
        m.i = a.perm ? (int64_t)a.perm[s] : (s < a.nrows ? s : -1);
        const uint32_t cidx = a.log2C >= 0 ? (uint32_t)s >> a.log2C : (uint32_t)s / (uint32_t)a.C;
        m.off = a.chunkptr[cidx] + (int64_t)((uint32_t)s - cidx * (uint32_t)a.C);
        m.len = a.slotlen[s];
        // without chunk lengths each lane runs to its own length (same sums)
        m.clen = (LS && a.chunklen) ? a.chunklen[cidx] : m.len;
        return m;
    };

    auto slot = [&](const Meta &m) {
        const int64_t i = m.i;
        if (i < 0) return;
        const int64_t off = m.off;
        const int len = m.len;
        // the epilogue's own loads (x_i, old y) go out before the row loop
        const bool epi_lane = (!MT || tt == 0) && nvalid > 0;
        XT xi[CPL], yo[CPL], t[CPL];
        XT *yp = y + i * a.yrs + (int64_t)k0 * a.ycs;
        if (early_epi && epi_lane) {
            if (need_xi) load_cols<XT, CPL, VEC>(xk + i * a.xrs, a.xcs, nvalid, xi);
            if (do_axpby) load_out<XT, CPL, VEC>(yp, a.ycs, nvalid, yo);
        }
        const int len_t = len > tt ? (len - tt + T - 1) >> lt : 0;
        XT rs[CPL];  // the row sums, in the vector precision
        {
            AT acc[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[c] = AT(0);
            int bad = 0;
            if constexpr (LS)
                row_product_ls<VT, XT, AT, CPL, VEC, U, false, ST>(val + off + (int64_t)tt * a.C,
                                                                   a.col + off + (int64_t)tt * a.C, a.C << lt, len_t,
                                                                   (m.clen + T - 1) >> lt, xk, a.xrs, a.xcs, nvalid,
                                                                   acc, bad);
            else if constexpr (pipe)
                row_product_pipe<VT, XT, AT, CPL, VEC, U, false, ST>(val + off + (int64_t)tt * a.C,
                                                                     a.col + off + (int64_t)tt * a.C, a.C << lt,
                                                                     len_t, xk, a.xrs, a.xcs, nvalid, acc, bad);
            else
                row_product<VT, XT, AT, CPL, VEC, U, false, ST>(val + off + (int64_t)tt * a.C,
                                                                a.col + off + (int64_t)tt * a.C, a.C << lt, len_t, xk,
                                                                a.xrs, a.xcs, nvalid, acc, bad);
            if constexpr (std::is_same<AT, float>::value && std::is_same<XT, double>::value) {
                // an x element outside the fast conversion's range: this lane's
                // share of the row again, with the conversion instruction
                if (bad) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) acc[c] = AT(0);
                    row_product<VT, XT, AT, CPL, VEC, U, true, ST>(val + off + (int64_t)tt * a.C,
                                                               a.col + off + (int64_t)tt * a.C, a.C << lt, len_t, xk,
                                                               a.xrs, a.xcs, nvalid, acc, bad);
                }
            }
            if (MT && T > 1) {
                // combine the T partial sums of the row (fixed xor tree)
#pragma unroll
                for (int c = 0; c < CPL; ++c)
                    for (int o = G; o < G * T; o <<= 1) acc[c] += __shfl_xor_sync(rowmask, acc[c], o);
                if (tt != 0) return;
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) rs[c] = acc_to_x<XT, AT>(acc[c]);
        }
        if (nvalid <= 0) return;
        if (!early_epi) {
            if (need_xi) load_cols<XT, CPL, VEC>(xk + i * a.xrs, a.xcs, nvalid, xi);
            if (do_axpby) load_out<XT, CPL, VEC>(yp, a.ycs, nvalid, yo);
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            XT v = rs[c];
            if constexpr (EPI == 3) {
                // beta = 1: y = alpha t - (alpha gamma) x_i + y_old as two fused
                // multiply-adds; the launcher passes alpha gamma (rounded once
                // on the host) in place of gamma
                v = fma_rn(alpha, v, fma_rn(-gam[c], xi[c], yo[c]));
            } else {
                if (shift) v = fma_rn(-gam[c], xi[c], v);
                if (do_scale) v = mul_rn(alpha, v);
                if (do_axpby) v = fma_rn(beta, yo[c], v);
            }
            t[c] = v;
        }
        // without the beta term y is not read by this call: streaming stores
        if (SP_STORE_CS_PLAIN != 0 && !do_axpby)
            store_out<XT, CPL, VEC, true>(yp, a.ycs, nvalid, t);
        else
            store_out<XT, CPL, VEC, false>(yp, a.ycs, nvalid, t);
        if constexpr (DOTS) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                if (c < nvalid) {
                    const DT td = (DT)t[c], xd = need_xi ? (DT)xi[c] : DT(0);
                    if constexpr ((DM & 1) != 0)
                        if (f & SP_SPMV_DOT_YY) dyy[c] = fma_rn(td, td, dyy[c]);
                    if constexpr ((DM & 2) != 0)
                        if (f & SP_SPMV_DOT_XY) dxy[c] = fma_rn(xd, td, dxy[c]);
                    if constexpr ((DM & 4) != 0)
                        if (f & SP_SPMV_DOT_XX) dxx[c] = fma_rn(xd, xd, dxx[c]);
                }
            }
        }
        if (do_chain) {
            XT zo[CPL];
            XT *zp = z + i * a.zrs + (int64_t)k0 * a.zcs;
            load_out<XT, CPL, VEC>(zp, a.zcs, nvalid, zo);
#pragma unroll
            for (int c = 0; c < CPL; ++c) zo[c] = fma_rn(eta, t[c], mul_rn(delta, zo[c]));
            store_out<XT, CPL, VEC>(zp, a.zcs, nvalid, zo);
        }
        if constexpr (MV > 0) {
            const double *__restrict__ vr = a.vty_V + i * a.vty_ldv;
            auto add = [&](int p, double vv) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) vacc[p][c] = fma_rn(vv, (double)t[c], vacc[p][c]);
            };
            // pairs measured faster for m <= 4 (231 -> 228 us at m = 4) and
            // slower at m = 8 (260 -> 263 us: more registers live)
            if (MV >= 2 && MV <= 4 && SP_VTY_VEC2 != 0 && a.vty_vec2) {
#pragma unroll
                for (int p = 0; p + 1 < MV; p += 2) {
                    if (p + 1 < a.vty_m) {
                        const double2 v2 = __ldg(reinterpret_cast<const double2 *>(vr + p));
                        add(p, v2.x);
                        add(p + 1, v2.y);
                    } else if (p < a.vty_m) {
                        add(p, __ldg(vr + p));
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < MV; ++p)
                    if (p < a.vty_m) add(p, __ldg(vr + p));
            }
        }
    };

    if constexpr (DM == 0 && MV == 0) {
        if (a.dyn_grab > 0) {
            // dynamic order (products without fused reductions, whose results do
            // not depend on which warp computes which rows): each warp takes the
            // next run of dyn_grab slots from a counter until none is left; the
            // last warp to finish resets the counter for the next launch
            unsigned *next = a.ticket + 1, *done = a.ticket + 2;
            const int64_t nruns = (a.nslots + a.dyn_grab - 1) / a.dyn_grab;
            for (;;) {
                unsigned r = 0;
                if (lane == 0) r = atomicAdd(next, 1u);
                r = __shfl_sync(0xffffffffu, r, 0);
                if ((int64_t)r >= nruns) break;
                const int64_t s0 = (int64_t)r * a.dyn_grab;
                const int64_t s1 = s0 + a.dyn_grab < a.nslots ? s0 + a.dyn_grab : a.nslots;
                for (int64_t s = s0 + rw; s < s1; s += Rr) slot(meta_of(s));
            }
            __threadfence();
            if (lane == 0 && atomicAdd(done, 1u) == gridDim.x * (unsigned)kMainWarps - 1u) {
                *next = 0u;
                *done = 0u;
            }
            return;
        }
    }
    if (a.sched) {
        // moving front: in round r this warp takes one 32-slot block of the
        // run of adjacent blocks the whole grid covers in that round
        const int64_t W = (int64_t)gridDim.x * kMainWarps;
        const int64_t me = (int64_t)blockIdx.x * kMainWarps + warp;
        int kb = a.sched[me];
        for (int r = 0; r < a.sched_rounds; ++r) {
            const int knext = r + 1 < a.sched_rounds ? a.sched[(int64_t)(r + 1) * W + me] : -1;
            if (kb >= 0) {
                const int64_t s0 = (int64_t)kb * 32;
                const int64_t s1 = s0 + 32 < a.nslots ? s0 + 32 : a.nslots;
                if constexpr (BANK) {
                    // every lane runs the same iterations (dot_tick is warp-wide)
                    for (int64_t sb = s0; sb < s1; sb += Rr) {
                        if (sb + rw < s1) slot(meta_of(sb + rw));
                        dot_tick();
                    }
                } else {
                    for (int64_t s = s0 + rw; s < s1; s += Rr) slot(meta_of(s));
                }
            }
            kb = knext;
        }
    } else if (a.wbounds) {
        // static cost-balanced partition: this warp owns a contiguous slot range
#if SP_SWIZZLE
        const int nsm = a.nsm, per = gridDim.x / nsm;
        const int bsw = (blockIdx.x % nsm) * per + blockIdx.x / nsm;
        const int gw = bsw * kMainWarps + warp;
#else
        const int gw = blockIdx.x * kMainWarps + warp;
#endif
        const int64_t s0 = (int64_t)a.wbounds[gw] * 32;
        const int64_t s1e = (int64_t)a.wbounds[gw + 1] * 32;
        const int64_t s1 = s1e < a.nslots ? s1e : a.nslots;
        int64_t s = s0 + rw;
        if (prefetch_meta && BANK) {
            // the next slot's metadata is loaded while this slot is computed;
            // the loop runs the same iterations in every lane (dot_tick is warp-wide)
            Meta cur{-1, 0, 0, -1};
            if (s < s1) cur = meta_of(s);
            for (int64_t sb = s0; sb < s1; sb += Rr, s += Rr) {
                Meta nxt{-1, 0, 0, -1};
                if (s + Rr < s1) nxt = meta_of(s + Rr);
                slot(cur);
                dot_tick();
                cur = nxt;
            }
        } else if (prefetch_meta) {
            Meta cur{-1, 0, 0, -1};
            if (s < s1) cur = meta_of(s);
            for (; s < s1; s += Rr) {
                Meta nxt{-1, 0, 0, -1};
                if (s + Rr < s1) nxt = meta_of(s + Rr);
                slot(cur);
                cur = nxt;
            }
        } else if constexpr (BANK) {
            for (int64_t sb = s0; sb < s1; sb += Rr, s += Rr) {
                if (s < s1) slot(meta_of(s));
                dot_tick();
            }
        } else {
            for (; s < s1; s += Rr) slot(meta_of(s));
        }
    } else {
        const int rows = Rr * kMainWarps;
        for (int64_t base = (int64_t)blockIdx.x * rows; base < a.nslots; base += (int64_t)gridDim.x * rows) {
            const int64_t s = base + warp * Rr + rw;
            if (s < a.nslots) slot(meta_of(s));
            dot_tick();
        }
    }
    if constexpr (DOTS) {
        double vyy[CPL], vxy[CPL], vxx[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            vyy[c] = (DM & 1) ? (double)dyy[(DM & 1) ? c : 0] : 0.0;
            vxy[c] = (DM & 2) ? (double)dxy[(DM & 2) ? c : 0] : 0.0;
            vxx[c] = (DM & 4) ? (double)dxx[(DM & 4) ? c : 0] : 0.0;
        }
        reduce_dots<CPL, G, DM, BANK>(a, k0, vyy, vxy, vxx);
    }
    if constexpr (MV > 0) reduce_vty<CPL, G, MV>(a, k0, vacc);
}

// Host-side dispatch over the block width for one (value, vector) type pair.
template <class VT, class XT>
int launch_spmv_typed(const SpmvArgs &a, bool vec, int max_blocks, cudaStream_t s);

}  // namespace sp
