// CSR -> SELL-C-sigma construction on the device (GHOST, Sec. "Sparse matrix
// storage": chunks of C rows padded to the chunk's longest row and stored
// column-wise; rows sorted by nonzero count inside windows of sigma rows).
//
// Steps, all as kernels on the caller's stream:
//   1. validate the CSR and take row lengths (a1)
//   2. stable descending sort of the row lengths inside every sigma window by
//      bottom-up merging of sorted runs (a2); each element finds its output
//      position with one binary search in the neighbouring run, so a pass is
//      one fully parallel kernel and ties keep the original row order
//   3. per-slot lengths, chunk lengths, chunk offsets by an int64 scan (a2)
//   4. scatter of column indices and values into chunk-column-major order (a3)
// The transpose (for the adjoint) is built the same way from the CSR of A^T,
// which comes from a stable ascending merge sort of the entries by column.
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"

namespace sp {

static constexpr int kThreads = 256;

static inline int grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535 * 32) g = 65535 * 32;
    return (int)g;
}

DevBuf::~DevBuf() {
    if (ptr) cudaFree(ptr);
}

int dev_alloc(DevBufPtr &out, size_t bytes, cudaStream_t) {
    auto b = std::make_shared<DevBuf>();
    if (bytes) {
        cudaError_t e = cudaMalloc(&b->ptr, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA;
        }
    }
    b->bytes = bytes;
    out = b;
    return SP_OK;
}


// ------------------------------------------------------------------ value rounding

template <class D>
__device__ __forceinline__ D cvt_from_double(double v);
template <>
__device__ __forceinline__ double cvt_from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ float cvt_from_double<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_double<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn(__double2float_rn(v));  // f64 -> f32 -> bf16, both RNE
}

template <class S>
__device__ __forceinline__ double to_double(S v) { return (double)v; }
template <>
__device__ __forceinline__ double to_double<__nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}

// ------------------------------------------------------------------ 1. validation

__global__ void k_validate_rows(const int64_t *__restrict__ rowptr, int64_t N, int64_t nnz,
                                int *__restrict__ err, int *__restrict__ maxlen,
                                int32_t *__restrict__ rowlen) {
    int local_max = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        if (i == 0 && a != 0) atomicOr(err, 1);
        if (i == N - 1 && b != nnz) atomicOr(err, 2);
        if (a > b || a < 0 || b > nnz || b - a > 0x7fffffff) {
            atomicOr(err, 4);
            rowlen[i] = 0;
        } else {
            int l = (int)(b - a);
            rowlen[i] = l;
            local_max = max(local_max, l);
        }
    }
    if (local_max) atomicMax(maxlen, local_max);
}

__global__ void k_validate_cols(const int32_t *__restrict__ col, int64_t nnz, int64_t ncols,
                                int *__restrict__ err) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = col[p];
        if (c < 0 || (int64_t)c >= ncols) atomicOr(err, 8);
    }
}

// ------------------------------------------------------------------ 2. windowed stable merge sort

__global__ void k_iota(int32_t *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

// One bottom-up merge pass: runs of length `run` (sorted) are merged pairwise
// inside windows of `window` elements.  DESC: larger keys first.  Stable:
// on equal keys the element of the left run comes first.
template <bool DESC>
__global__ void k_merge_pass(const int32_t *__restrict__ ks, const int32_t *__restrict__ vs,
                             int32_t *__restrict__ kd, int32_t *__restrict__ vd, int64_t n,
                             int64_t window, int64_t run) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t w0 = (e / window) * window;
        int64_t w1 = min(w0 + window, n);
        int64_t o = e - w0;
        int64_t p0 = w0 + (o / (2 * run)) * (2 * run);
        int64_t mid = min(p0 + run, w1);
        int64_t end = min(p0 + 2 * run, w1);
        int32_t key = ks[e];
        int64_t out;
        if (e < mid) {
            // how many right-run elements precede this left element:
            // those strictly before it in the order (DESC: key_b > key)
            int64_t lo = mid, hi = end;
            while (lo < hi) {
                int64_t m = (lo + hi) >> 1;
                bool before = DESC ? (ks[m] > key) : (ks[m] < key);
                if (before) lo = m + 1; else hi = m;
            }
            out = e + (lo - mid);  // = p0 + (e - p0) + (lo - mid)
        } else {
            // left-run elements that precede a right element: those not after it
            // (DESC: key_a >= key), ties from the left go first
            int64_t lo = p0, hi = mid;
            while (lo < hi) {
                int64_t m = (lo + hi) >> 1;
                bool before = DESC ? (ks[m] >= key) : (ks[m] <= key);
                if (before) lo = m + 1; else hi = m;
            }
            out = p0 + (e - mid) + (lo - p0);
        }
        kd[out] = key;
        vd[out] = vs[e];
    }
}

// Stable sort of (key, value) int32 pairs inside windows; result in (k0, v0).
template <bool DESC>
static int windowed_sort(int32_t *k0, int32_t *v0, int32_t *k1, int32_t *v1, int64_t n, int64_t window,
                         cudaStream_t s) {
    int64_t lim = std::min<int64_t>(window, n);
    bool in0 = true;
    for (int64_t run = 1; run < lim; run *= 2) {
        if (in0)
            k_merge_pass<DESC><<<grid_for(n), kThreads, 0, s>>>(k0, v0, k1, v1, n, window, run);
        else
            k_merge_pass<DESC><<<grid_for(n), kThreads, 0, s>>>(k1, v1, k0, v0, n, window, run);
        in0 = !in0;
    }
    SP_CUDA(cudaGetLastError());
    if (!in0) {
        SP_CUDA(cudaMemcpyAsync(k0, k1, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        SP_CUDA(cudaMemcpyAsync(v0, v1, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    return SP_OK;
}

// ------------------------------------------------------------------ 3. slots, chunks, scan

__global__ void k_slots(const int32_t *__restrict__ sorted_len, const int32_t *__restrict__ sorted_row,
                        int64_t N, int64_t nslots, int32_t *__restrict__ slotlen,
                        int32_t *__restrict__ perm) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
         s += (int64_t)gridDim.x * blockDim.x) {
        bool real = s < N;
        slotlen[s] = real ? sorted_len[s] : 0;
        perm[s] = real ? sorted_row[s] : -1;
    }
}

__global__ void k_chunklen(const int32_t *__restrict__ slotlen, int64_t nch, int C,
                           int32_t *__restrict__ chunklen, int64_t *__restrict__ chunksize) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = 0;
        for (int r = 0; r < C; ++r) m = max(m, slotlen[c * C + r]);
        chunklen[c] = m;
        chunksize[c] = (int64_t)C * m;
    }
}

// Exclusive int64 scan: blocks of 1024 threads x 4 elements, block totals
// scanned recursively, then added back.
static constexpr int kScanThreads = 1024;
static constexpr int kScanItems = 4;
static constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan_tile(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
            int64_t *__restrict__ totals) {
    __shared__ int64_t warp_sums[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = base + q < n ? in[base + q] : 0;
        sum += v[q];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t ws = warp_sums[lane];
        int64_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - ws;  // exclusive
        if (lane == 31 && totals) totals[blockIdx.x] = wi;
    }
    __syncthreads();
    int64_t run = warp_sums[wid] + inc - sum;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t add = offs[blockIdx.x];
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < n) out[base + t] += add;
}

static int scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return SP_OK;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        SP_CUDA(cudaGetLastError());
        return SP_OK;
    }
    Tmp tot(s), totx(s);
    SP_TRY(tot.alloc(nb * sizeof(int64_t)));
    SP_TRY(totx.alloc(nb * sizeof(int64_t)));
    k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tot.as<int64_t>());
    SP_CUDA(cudaGetLastError());
    SP_TRY(scan_exclusive(tot.as<int64_t>(), totx.as<int64_t>(), nb, s));
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, totx.as<int64_t>());
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------ 4. scatter into SELL order

// Slot s = c*C + r holds original row perm[s]; its entry j goes to
// chunkptr[c] + j*C + r.  Padding: column of the row's last entry (0 for an
// empty or padding row); values are written by k_fill_values.
// colmap (may be null): column index map applied to every stored index (the
// slot of each row, for matrices whose vectors live in SELL row order)
__global__ void k_scatter_cols(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ perm, const int32_t *__restrict__ chunklen,
                               const int64_t *__restrict__ chunkptr, int64_t nslots, int C,
                               const int32_t *__restrict__ colmap, int32_t *__restrict__ col_sell) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = s / C;
        int r = (int)(s - c * C);
        int32_t i = perm[s];
        int64_t start = i >= 0 ? rowptr[i] : 0;
        int64_t len = i >= 0 ? rowptr[i + 1] - start : 0;
        int32_t pad = len > 0 ? col[start + len - 1] : 0;
        int64_t base = chunkptr[c] + r;
        int32_t cl = chunklen[c];
        if (colmap && len > 0) pad = colmap[pad];
        for (int64_t j = 0; j < cl; ++j) {
            int32_t v = pad;
            if (j < len) v = colmap ? colmap[col[start + j]] : col[start + j];
            col_sell[base + j * C] = v;
        }
    }
}

// inv[perm[s]] = s for the real slots (s < nrows)
__global__ void k_invert_perm(const int32_t *__restrict__ perm, int64_t nrows, int32_t *__restrict__ inv) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nrows;
         s += (int64_t)gridDim.x * blockDim.x)
        inv[perm[s]] = (int32_t)s;
}

template <class S, class D>
__global__ void k_fill_values(const int64_t *__restrict__ rowptr, const S *__restrict__ val,
                              const int32_t *__restrict__ perm, const int32_t *__restrict__ chunklen,
                              const int64_t *__restrict__ chunkptr, int64_t nslots, int C,
                              D *__restrict__ val_sell) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = s / C;
        int r = (int)(s - c * C);
        int32_t i = perm[s];
        int64_t start = i >= 0 ? rowptr[i] : 0;
        int64_t len = i >= 0 ? rowptr[i + 1] - start : 0;
        int64_t base = chunkptr[c] + r;
        int32_t cl = chunklen[c];
        for (int64_t j = 0; j < cl; ++j)
            val_sell[base + j * C] = cvt_from_double<D>(j < len ? (double)val[start + j] : 0.0);
    }
}

template <class S>
static void launch_fill(const Pattern &P, sp_dtype vdt, void *out, const S *in, cudaStream_t s) {
    const int64_t *rp = (const int64_t *)P.rowptr->ptr;
    const int32_t *pm = (const int32_t *)P.perm->ptr;
    const int32_t *cl = (const int32_t *)P.chunklen->ptr;
    const int64_t *cp = (const int64_t *)P.chunkptr->ptr;
    int g = grid_for(P.nslots);
    if (vdt == SP_F64)
        k_fill_values<S, double><<<g, kThreads, 0, s>>>(rp, in, pm, cl, cp, P.nslots, P.C, (double *)out);
    else if (vdt == SP_F32)
        k_fill_values<S, float><<<g, kThreads, 0, s>>>(rp, in, pm, cl, cp, P.nslots, P.C, (float *)out);
    else
        k_fill_values<S, __nv_bfloat16>
            <<<g, kThreads, 0, s>>>(rp, in, pm, cl, cp, P.nslots, P.C, (__nv_bfloat16 *)out);
}

int fill_values_from_csr(const Pattern &P, sp_dtype vdt, void *val_sell, const void *d_val_csr,
                         bool val_f32, cudaStream_t s) {
    if (P.nslots == 0) return SP_OK;
    if (val_f32)
        launch_fill<float>(P, vdt, val_sell, (const float *)d_val_csr, s);
    else
        launch_fill<double>(P, vdt, val_sell, (const double *)d_val_csr, s);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

// ------------------------------------------------------------------ static work partition

// cost of each 32-slot block: stored-entry work of its rows + SP_ROW_COST per
// real row (the epilogue and the fixed latency of a row); slots >= nrows are
// padding rows
#ifndef SP_ROW_COST
#define SP_ROW_COST 16
#endif
__global__ void k_block32_cost(const int32_t *__restrict__ slotlen, int64_t nslots, int64_t nrows,
                               int64_t nb32, int64_t *__restrict__ cost) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb32;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        int64_t e = min(32 * k + 32, nslots);
        for (int64_t s = 32 * k; s < e; ++s) c += slotlen[s] + (s < nrows ? SP_ROW_COST : 0);
        cost[k] = c;
    }
}

// per 32-slot block: longest and shortest real row; out[0] += longest -
// shortest, out[1] += longest (one atomic per warp)
__global__ void k_block_spread(const int32_t *__restrict__ slotlen, int64_t nslots, int64_t nrows, int64_t nb32,
                               unsigned long long *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t kend = (nb32 + 31) / 32 * 32;  // whole warps run every iteration
    for (int64_t k = k0; k < kend; k += stride) {
        unsigned long long d = 0, m = 0;
        if (k < nb32) {
            int lo = INT_MAX, hi = 0;
            const int64_t e = min(32 * k + 32, min(nslots, nrows));
            for (int64_t s = 32 * k; s < e; ++s) {
                lo = min(lo, slotlen[s]);
                hi = max(hi, slotlen[s]);
            }
            if (hi > 0) {
                d = (unsigned long long)(hi - lo);
                m = (unsigned long long)hi;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d += __shfl_xor_sync(0xffffffffu, d, o);
            m += __shfl_xor_sync(0xffffffffu, m, o);
        }
        if ((threadIdx.x & 31) == 0 && m > 0) {
            atomicAdd(out, d);
            atomicAdd(out + 1, m);
        }
    }
}

// bounds[t] = first block whose prefix cost reaches t/T of the total
__global__ void k_partition(const int64_t *__restrict__ prefix, int64_t nb32, int64_t T,
                            int32_t *__restrict__ bounds) {
    int64_t total = prefix[nb32];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t k;
        if (t == 0) {
            k = 0;
        } else if (t == T) {
            k = nb32;
        } else {
            int64_t target = (total * t + T / 2) / T;
            int64_t lo = 0, hi = nb32;
            while (lo < hi) {
                int64_t m = (lo + hi) >> 1;
                if (prefix[m] < target) lo = m + 1; else hi = m;
            }
            k = lo;
        }
        bounds[t] = (int32_t)k;
    }
}

// Stable insertion sort of a short array (the 32 blocks or warps of one CTA):
// the same order as std::stable_sort, without its temporary buffer.
template <class Less>
static void stable_small_sort(int32_t *a, int n, Less less) {
    for (int i = 1; i < n; ++i) {
        const int32_t v = a[i];
        int j = i;
        while (j > 0 && less(v, a[j - 1])) {
            a[j] = a[j - 1];
            --j;
        }
        a[j] = v;
    }
}

int build_partition(Pattern &P, cudaStream_t s) {
    int sms = 1;
    SP_TRY(device_sm_count(&sms));
    int64_t nb32 = (P.nslots + 31) / 32;
    if (nb32 >= (1LL << 31)) return SP_OK;
    Tmp cost(s), prefix(s);
    SP_TRY(cost.alloc((nb32 + 1) * sizeof(int64_t)));
    SP_TRY(prefix.alloc((nb32 + 1) * sizeof(int64_t)));
    SP_CUDA(cudaMemsetAsync(cost.p, 0, (nb32 + 1) * sizeof(int64_t), s));
    if (nb32 > 0) {
        k_block32_cost<<<grid_for(nb32), kThreads, 0, s>>>((const int32_t *)P.slotlen->ptr, P.nslots, P.nrows,
                                                            nb32, cost.as<int64_t>());
        SP_CUDA(cudaGetLastError());
    }
    SP_TRY(scan_exclusive(cost.as<int64_t>(), prefix.as<int64_t>(), nb32 + 1, s));
    if (nb32 > 0) {
        Tmp spread(s);
        SP_TRY(spread.alloc(2 * sizeof(unsigned long long)));
        SP_CUDA(cudaMemsetAsync(spread.p, 0, 2 * sizeof(unsigned long long), s));
        k_block_spread<<<grid_for(nb32), kThreads, 0, s>>>((const int32_t *)P.slotlen->ptr, P.nslots, P.nrows, nb32,
                                                            (unsigned long long *)spread.p);
        SP_CUDA(cudaGetLastError());
        unsigned long long h[2] = {0, 0};
        SP_CUDA(cudaMemcpyAsync(h, spread.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        P.lane_spread = h[1] ? (double)h[0] / (double)h[1] : 0.0;
    }
    int64_t total = 0;
    for (int b = 1; b <= kMaxOcc; ++b) {
        P.bounds_off[b] = total;
        total += (int64_t)kPartWarps * b * sms + 1;
    }
    SP_TRY(dev_alloc(P.bounds, total * sizeof(int32_t), s));
    for (int b = 1; b <= kMaxOcc; ++b) {
        int64_t T = (int64_t)kPartWarps * b * sms;
        k_partition<<<grid_for(T + 1), kThreads, 0, s>>>(prefix.as<int64_t>(), nb32, T,
                                                          (int32_t *)P.bounds->ptr + P.bounds_off[b]);
        SP_CUDA(cudaGetLastError());
    }
    P.bounds_sms = sms;

    // moving-front schedule, for the grid the product kernel runs: one
    // resident kSchedCtaWarps-warp CTA per SM (every product kernel holds 56 to
    // 64 registers per thread at 1024 threads, so a second CTA never fits; a
    // grid without a table takes the contiguous ranges instead).  Building
    // the table for two CTAs per SM as well cost about 3.5 ms of host time per
    // matrix of 2M rows.
    if (nb32 > 0) {
        std::vector<int64_t> c(nb32);
        SP_CUDA(cudaMemcpyAsync(c.data(), cost.p, nb32 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SP_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> table;
        for (int b = 1; b <= kMaxOcc; ++b) {
            const int64_t W = (int64_t)kPartWarps * b * sms;
            if (b * kPartWarps != kSchedCtaWarps * kSchedResidentCtas) continue;
            const int64_t rounds = (nb32 + W - 1) / W;
            P.sched_off[b] = (int64_t)table.size();
            P.sched_rounds[b] = (int32_t)rounds;
            table.resize(table.size() + rounds * W, -1);
            int32_t *t = table.data() + P.sched_off[b];
            // each round covers W adjacent blocks in runs of kSchedCtaWarps;
            // the runs go to CTAs longest first, each to the CTA with the least
            // work so far (so sorted rows do not load the low CTAs every round),
            // and inside a CTA the blocks go to warps the same way
            const int64_t nct = W / kSchedCtaWarps;
            std::vector<int64_t> load(W, 0), cload(nct, 0), rcost(nct);
            std::vector<int32_t> run(nct), ctas(nct);
            int32_t blk[kSchedCtaWarps], wrp[kSchedCtaWarps];
            for (int64_t r = 0; r < rounds; ++r) {
                for (int64_t g = 0; g < nct; ++g) {
                    run[g] = (int32_t)g;
                    ctas[g] = (int32_t)g;
                    rcost[g] = 0;
                    for (int64_t j = r * W + g * kSchedCtaWarps; j < r * W + (g + 1) * kSchedCtaWarps && j < nb32; ++j)
                        rcost[g] += c[j];
                }
                std::stable_sort(run.begin(), run.end(), [&](int32_t x, int32_t y) { return rcost[x] > rcost[y]; });
                std::stable_sort(ctas.begin(), ctas.end(), [&](int32_t x, int32_t y) { return cload[x] < cload[y]; });
                for (int64_t q = 0; q < nct; ++q) {
                    const int64_t cta = ctas[q];
                    const int64_t first = r * W + (int64_t)run[q] * kSchedCtaWarps;
                    cload[cta] += rcost[run[q]];
                    int n = 0;
                    for (int j = 0; j < kSchedCtaWarps && first + j < nb32; ++j) blk[n++] = (int32_t)(first + j);
                    if (!n) continue;
                    int64_t *ld = load.data() + cta * kSchedCtaWarps;
                    for (int j = 0; j < kSchedCtaWarps; ++j) wrp[j] = j;
                    stable_small_sort(blk, n, [&](int32_t x, int32_t y) { return c[x] > c[y]; });
                    stable_small_sort(wrp, kSchedCtaWarps, [&](int32_t x, int32_t y) { return ld[x] < ld[y]; });
                    for (int i = 0; i < n; ++i) {
                        t[r * W + cta * kSchedCtaWarps + wrp[i]] = blk[i];
                        ld[wrp[i]] += c[blk[i]];
                    }
                }
            }
        }
        if (!table.empty()) {
            SP_TRY(dev_alloc(P.sched, table.size() * sizeof(int32_t), s));
            SP_CUDA(cudaMemcpyAsync(P.sched->ptr, table.data(), table.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
            SP_CUDA(cudaStreamSynchronize(s));
        }
    }
    return SP_OK;
}

// ------------------------------------------------------------------ whole construction

int build_pattern_and_values(sp_mat *A, int64_t N, int64_t ncols, const int64_t *d_rowptr,
                             const int32_t *d_col, const void *d_val, bool val_f32, int C,
                             int64_t sigma, cudaStream_t s, bool permuted) {
    auto P = std::make_shared<Pattern>();
    P->nrows = N;
    P->ncols = ncols;
    P->C = C;
    P->sigma = sigma;
    int64_t nnz = 0;
    if (N > 0) SP_CUDA(cudaMemcpyAsync(&nnz, d_rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    if (nnz < 0) return SP_ERR_FORMAT;
    P->nnz = nnz;
    P->nchunks = (N + C - 1) / C;
    P->nslots = P->nchunks * C;

    // 1. validation + row lengths
    Tmp flags(s), rowlen(s);
    SP_TRY(flags.alloc(2 * sizeof(int)));
    SP_TRY(rowlen.alloc((N + 1) * sizeof(int32_t)));
    SP_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s));
    if (N > 0) {
        k_validate_rows<<<grid_for(N), kThreads, 0, s>>>(d_rowptr, N, nnz, flags.as<int>(),
                                                         flags.as<int>() + 1, rowlen.as<int32_t>());
        SP_CUDA(cudaGetLastError());
    }
    if (nnz > 0) {
        k_validate_cols<<<grid_for(nnz), kThreads, 0, s>>>(d_col, nnz, ncols, flags.as<int>());
        SP_CUDA(cudaGetLastError());
    }
    int hflags[2] = {0, 0};
    SP_CUDA(cudaMemcpyAsync(hflags, flags.p, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    if (hflags[0]) return SP_ERR_FORMAT;
    P->maxrowlen = hflags[1];

    // keep the CSR row pointers (value updates, sampled products, CSR export)
    SP_TRY(dev_alloc(P->rowptr, (N + 1) * sizeof(int64_t), s));
    SP_CUDA(cudaMemcpyAsync(P->rowptr->ptr, d_rowptr, (N + 1) * sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, s));

    // 2. sigma-window sort (descending, stable)
    Tmp k1(s), v0(s), v1(s);
    SP_TRY(k1.alloc((N + 1) * sizeof(int32_t)));
    SP_TRY(v0.alloc((N + 1) * sizeof(int32_t)));
    SP_TRY(v1.alloc((N + 1) * sizeof(int32_t)));
    if (N > 0) {
        k_iota<<<grid_for(N), kThreads, 0, s>>>(v0.as<int32_t>(), N);
        SP_CUDA(cudaGetLastError());
        if (sigma > 1)
            SP_TRY(windowed_sort<true>(rowlen.as<int32_t>(), v0.as<int32_t>(), k1.as<int32_t>(),
                                       v1.as<int32_t>(), N, sigma, s));
    }

    // 3. slots and chunks
    SP_TRY(dev_alloc(P->slotlen, P->nslots * sizeof(int32_t), s));
    SP_TRY(dev_alloc(P->perm, P->nslots * sizeof(int32_t), s));
    SP_TRY(dev_alloc(P->chunklen, P->nchunks * sizeof(int32_t), s));
    SP_TRY(dev_alloc(P->chunkptr, (P->nchunks + 1) * sizeof(int64_t), s));
    if (P->nslots > 0) {
        k_slots<<<grid_for(P->nslots), kThreads, 0, s>>>(rowlen.as<int32_t>(), v0.as<int32_t>(), N,
                                                          P->nslots, (int32_t *)P->slotlen->ptr,
                                                          (int32_t *)P->perm->ptr);
        SP_CUDA(cudaGetLastError());
    }
    Tmp sizes(s);
    SP_TRY(sizes.alloc((P->nchunks + 1) * sizeof(int64_t)));
    SP_CUDA(cudaMemsetAsync(sizes.p, 0, (P->nchunks + 1) * sizeof(int64_t), s));
    if (P->nchunks > 0) {
        k_chunklen<<<grid_for(P->nchunks), kThreads, 0, s>>>((const int32_t *)P->slotlen->ptr, P->nchunks,
                                                              C, (int32_t *)P->chunklen->ptr,
                                                              sizes.as<int64_t>());
        SP_CUDA(cudaGetLastError());
    }
    SP_TRY(scan_exclusive(sizes.as<int64_t>(), (int64_t *)P->chunkptr->ptr, P->nchunks + 1, s));
    int64_t nstored = 0;
    SP_CUDA(cudaMemcpyAsync(&nstored, (int64_t *)P->chunkptr->ptr + P->nchunks, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
    SP_CUDA(cudaStreamSynchronize(s));
    P->nstored = nstored;

    // 4. scatter
    SP_TRY(dev_alloc(P->col, nstored * sizeof(int32_t), s));
    if (P->nslots > 0) {
        Tmp inv(s);
        const int32_t *colmap = nullptr;
        if (permuted) {
            SP_TRY(inv.alloc(std::max<int64_t>(N, 1) * sizeof(int32_t)));
            k_invert_perm<<<grid_for(std::max<int64_t>(N, 1)), kThreads, 0, s>>>((const int32_t *)P->perm->ptr, N,
                                                                              inv.as<int32_t>());
            SP_CUDA(cudaGetLastError());
            colmap = inv.as<int32_t>();
        }
        k_scatter_cols<<<grid_for(P->nslots), kThreads, 0, s>>>(
            d_rowptr, d_col, (const int32_t *)P->perm->ptr, (const int32_t *)P->chunklen->ptr,
            (const int64_t *)P->chunkptr->ptr, P->nslots, C, colmap, (int32_t *)P->col->ptr);
        SP_CUDA(cudaGetLastError());
        SP_CUDA(cudaStreamSynchronize(s));
    }
    P->permuted_space = permuted;
    SP_TRY(build_partition(*P, s));
    DevBufPtr val;
    SP_TRY(dev_alloc(val, nstored * dtype_size(A->vdt), s));
    SP_TRY(fill_values_from_csr(*P, A->vdt, val->ptr, d_val, val_f32, s));
    SP_CUDA(cudaStreamSynchronize(s));
    A->pat = P;
    A->val = val;
    return SP_OK;
}

// ------------------------------------------------------------------ transpose

__global__ void k_entry_rows(const int64_t *__restrict__ rowptr, int64_t N, int32_t *__restrict__ rowidx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) rowidx[p] = (int32_t)i;
}

// rowptr of A^T: number of entries with column < c, by binary search in the
// ascending sorted column keys.
__global__ void k_lower_bounds(const int32_t *__restrict__ keys, int64_t n, int64_t nout,
                               int64_t *__restrict__ out) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nout;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t m = (lo + hi) >> 1;
            if ((int64_t)keys[m] < c) lo = m + 1; else hi = m;
        }
        out[c] = lo;
    }
}

template <class V>
__global__ void k_transpose_entries(const int32_t *__restrict__ order, const int32_t *__restrict__ rowidx,
                                    const V *__restrict__ val, int64_t nnz, int32_t *__restrict__ colT,
                                    V *__restrict__ valT, int64_t *__restrict__ src) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = order[q];
        colT[q] = rowidx[p];
        valT[q] = val[p];
        src[q] = p;
    }
}

int build_transpose(sp_mat *A, const int64_t *d_rowptr, const int32_t *d_col, const void *d_val,
                    bool val_f32, cudaStream_t s) {
    const Pattern &P = *A->pat;
    int64_t nnz = P.nnz;
    if (nnz > 0x7fffffffLL) return SP_ERR_UNSUPPORTED;
    size_t vs = val_f32 ? 4 : 8;
    Tmp rowidx(s), k0(s), k1(s), v0(s), v1(s), rpT(s), colT(s), valT(s);
    SP_TRY(rowidx.alloc(nnz * 4));
    SP_TRY(k0.alloc(nnz * 4));
    SP_TRY(k1.alloc(nnz * 4));
    SP_TRY(v0.alloc(nnz * 4));
    SP_TRY(v1.alloc(nnz * 4));
    SP_TRY(rpT.alloc((P.ncols + 1) * 8));
    SP_TRY(colT.alloc(nnz * 4));
    SP_TRY(valT.alloc(nnz * vs));
    DevBufPtr src;
    SP_TRY(dev_alloc(src, nnz * sizeof(int64_t), s));
    if (nnz > 0) {
        k_entry_rows<<<grid_for(P.nrows), kThreads, 0, s>>>(d_rowptr, P.nrows, rowidx.as<int32_t>());
        SP_CUDA(cudaMemcpyAsync(k0.p, d_col, nnz * 4, cudaMemcpyDeviceToDevice, s));
        k_iota<<<grid_for(nnz), kThreads, 0, s>>>(v0.as<int32_t>(), nnz);
        SP_CUDA(cudaGetLastError());
        SP_TRY(windowed_sort<false>(k0.as<int32_t>(), v0.as<int32_t>(), k1.as<int32_t>(), v1.as<int32_t>(),
                                    nnz, nnz, s));
        if (val_f32)
            k_transpose_entries<float><<<grid_for(nnz), kThreads, 0, s>>>(
                v0.as<int32_t>(), rowidx.as<int32_t>(), (const float *)d_val, nnz, colT.as<int32_t>(),
                valT.as<float>(), (int64_t *)src->ptr);
        else
            k_transpose_entries<double><<<grid_for(nnz), kThreads, 0, s>>>(
                v0.as<int32_t>(), rowidx.as<int32_t>(), (const double *)d_val, nnz, colT.as<int32_t>(),
                valT.as<double>(), (int64_t *)src->ptr);
        SP_CUDA(cudaGetLastError());
    }
    k_lower_bounds<<<grid_for(P.ncols + 1), kThreads, 0, s>>>(k0.as<int32_t>(), nnz, P.ncols + 1,
                                                              rpT.as<int64_t>());
    SP_CUDA(cudaGetLastError());
    sp_mat *T = new sp_mat();
    T->vdt = A->vdt;
    int rc = build_pattern_and_values(T, P.ncols, P.nrows, rpT.as<int64_t>(), colT.as<int32_t>(), valT.p,
                                      val_f32, P.C, P.sigma, s);
    if (rc != SP_OK) {
        delete T;
        return rc;
    }
    T->pat->src_index = src;
    A->transpose = T;
    return SP_OK;
}

// ------------------------------------------------------------------ value gathers / conversions

template <class S, class D>
__global__ void k_gather(const S *__restrict__ src, const int64_t *__restrict__ index, int64_t n,
                         D *__restrict__ dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = (D)src[index[q]];
}

int gather_values(const void *src, bool src_f32, const int64_t *index, int64_t n, void *dst, bool dst_f32,
                  cudaStream_t s) {
    if (n <= 0) return SP_OK;
    if (src_f32 && dst_f32)
        k_gather<float, float><<<grid_for(n), kThreads, 0, s>>>((const float *)src, index, n, (float *)dst);
    else if (!src_f32 && !dst_f32)
        k_gather<double, double><<<grid_for(n), kThreads, 0, s>>>((const double *)src, index, n, (double *)dst);
    else
        return SP_ERR_ARG;
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

template <class S, class D>
__global__ void k_convert(const S *__restrict__ src, D *__restrict__ dst, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = cvt_from_double<D>(to_double<S>(src[q]));
}

template <class S>
static int convert_from(const S *src, void *dst, sp_dtype ddt, int64_t n, cudaStream_t s) {
    if (ddt == SP_F64)
        k_convert<S, double><<<grid_for(n), kThreads, 0, s>>>(src, (double *)dst, n);
    else if (ddt == SP_F32)
        k_convert<S, float><<<grid_for(n), kThreads, 0, s>>>(src, (float *)dst, n);
    else
        k_convert<S, __nv_bfloat16><<<grid_for(n), kThreads, 0, s>>>(src, (__nv_bfloat16 *)dst, n);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int convert_values(const void *src, sp_dtype sdt, void *dst, sp_dtype ddt, int64_t n, cudaStream_t s) {
    if (n <= 0) return SP_OK;
    if (sdt == SP_F64) return convert_from((const double *)src, dst, ddt, n, s);
    if (sdt == SP_F32) return convert_from((const float *)src, dst, ddt, n, s);
    return convert_from((const __nv_bfloat16 *)src, dst, ddt, n, s);
}

int widen_values(const void *src, sp_dtype sdt, double *dst, int64_t n, cudaStream_t s) {
    return convert_values(src, sdt, dst, SP_F64, n, s);
}

}  // namespace sp
