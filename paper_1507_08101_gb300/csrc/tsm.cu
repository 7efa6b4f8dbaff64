// Tall and skinny block-vector kernels (the dense-matrix section of the paper:
// V is n x m, W is n x k with m, k << n, X is m x k):
//     tsmttsm:  X <- alpha V^T W + beta X   (inner products of block vectors;
//               with a Kahan-compensated variant for large n)
//     tsmm:     W <- alpha V X + beta W      (also in place, W = V, k = m)
// Row-major blocks on the device, m, k <= 32.  Both stream V and W once.
//
// tsmttsm: each block takes a contiguous range of rows in tiles of kTileRows,
// staged in shared memory; each thread owns up to four of the m*k outputs and
// adds that tile's products into them.  The per-block sums go to a partial
// array and a second kernel adds them in block order, so the result does not
// depend on timing.  tsmm: each block stages a tile of rows of V, computes the
// tile's rows of the result from the small matrix in shared memory, and only
// then writes, so the in-place form reads every row before it overwrites it.
#include <algorithm>

#include "common.cuh"

namespace sp {

constexpr int kTsmThreads = 256;
constexpr int kTileRows = 32;
constexpr int kTsmMax = 32;
constexpr int kPerThread = kTsmMax * kTsmMax / kTsmThreads;  // outputs per thread (4)

template <class T, bool KAHAN>
__global__ void __launch_bounds__(kTsmThreads) k_tsmttsm_part(const T *__restrict__ V, int64_t ldv,
                                                              const T *__restrict__ W, int64_t ldw, int64_t n, int m,
                                                              int k, int64_t rows_per_block, double *__restrict__ part) {
    __shared__ T sv[kTileRows][kTsmMax], sw[kTileRows][kTsmMax];
    const int t = threadIdx.x;
    T acc[kPerThread], comp[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) acc[j] = comp[j] = T(0);
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = n < r0 + rows_per_block ? n : r0 + rows_per_block;
    const int mk = m * k;
    for (int64_t base = r0; base < r1; base += kTileRows) {
        const int rows = (int)(r1 - base < kTileRows ? r1 - base : kTileRows);
        for (int e = t; e < kTileRows * m; e += kTsmThreads) {
            const int r = e / m, c = e - r * m;
            sv[r][c] = r < rows ? V[(base + r) * ldv + c] : T(0);
        }
        for (int e = t; e < kTileRows * k; e += kTsmThreads) {
            const int r = e / k, c = e - r * k;
            sw[r][c] = r < rows ? W[(base + r) * ldw + c] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const int e = t + j * kTsmThreads;
            if (e < mk) {
                const int a = e / k, b = e - a * k;
                for (int r = 0; r < rows; ++r) {
                    const T p = sv[r][a] * sw[r][b];
                    if constexpr (KAHAN) {
                        // Kahan's compensated summation: comp carries the
                        // low-order part lost by the last addition
                        const T yv = p - comp[j];
                        const T tv = acc[j] + yv;
                        comp[j] = (tv - acc[j]) - yv;
                        acc[j] = tv;
                    } else {
                        acc[j] = fma(sv[r][a], sw[r][b], acc[j]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int e = t + j * kTsmThreads;
        if (e < mk) part[(int64_t)blockIdx.x * mk + e] = (double)acc[j] - (KAHAN ? (double)comp[j] : 0.0);
    }
}

// X[a, b] = alpha * sum over blocks (in block order) + beta X[a, b]
template <class T, bool KAHAN>
__global__ void k_tsmttsm_final(const double *__restrict__ part, int nblocks, int m, int k, double alpha,
                                double beta, T *__restrict__ X, int64_t ldx) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * k) return;
    double s = 0.0, c = 0.0;
    for (int bl = 0; bl < nblocks; ++bl) {
        const double p = part[(int64_t)bl * m * k + e];
        if constexpr (KAHAN) {
            const double yv = p - c;
            const double tv = s + yv;
            c = (tv - s) - yv;
            s = tv;
        } else {
            s += p;
        }
    }
    const int a = e / k, b = e - a * k;
    T *xp = X + (int64_t)a * ldx + b;
    const double old = beta != 0.0 ? (double)*xp : 0.0;
    *xp = (T)(alpha * s + beta * old);
}

template <class T>
__global__ void __launch_bounds__(kTsmThreads) k_tsmm(const T *__restrict__ V, int64_t ldv, const T *__restrict__ X,
                                                      int64_t ldx, T *W, int64_t ldw, int64_t n, int m, int k,
                                                      T alpha, T beta) {
    __shared__ T sx[kTsmMax][kTsmMax];
    __shared__ T sv[kTileRows][kTsmMax];
    const int t = threadIdx.x;
    for (int e = t; e < m * k; e += kTsmThreads) {
        const int a = e / k, b = e - a * k;
        sx[a][b] = X[(int64_t)a * ldx + b];
    }
    for (int64_t base = (int64_t)blockIdx.x * kTileRows; base < n; base += (int64_t)gridDim.x * kTileRows) {
        const int rows = (int)(n - base < kTileRows ? n - base : kTileRows);
        for (int e = t; e < kTileRows * m; e += kTsmThreads) {
            const int r = e / m, c = e - r * m;
            sv[r][c] = r < rows ? V[(base + r) * ldv + c] : T(0);
        }
        __syncthreads();  // the tile of V is read before W (which may be V) is written
        T out[kPerThread];
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const int e = t + j * kTsmThreads;
            out[j] = T(0);
            if (e < kTileRows * k) {
                const int r = e / k, b = e - r * k;
                if (r < rows) {
                    T s = T(0);
                    for (int a = 0; a < m; ++a) s = fma(sv[r][a], sx[a][b], s);
                    const T old = beta != T(0) ? W[(base + r) * ldw + b] : T(0);
                    out[j] = fma(alpha, s, beta * old);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const int e = t + j * kTsmThreads;
            if (e < kTileRows * k) {
                const int r = e / k, b = e - r * k;
                if (r < rows) W[(base + r) * ldw + b] = out[j];
            }
        }
    }
}

static int sms_blocks(int per_sm) {
    int sms = 1;
    device_sm_count(&sms);
    return sms * per_sm;
}

}  // namespace sp

using sp::DevBufPtr;

static bool rowmajor_dev(const sp_dense *d) { return d && d->layout == SP_ROW_MAJOR && d->ptr; }

int sp_tsmttsm(sp_dense *X, const sp_dense *V, const sp_dense *W, double alpha, double beta, int kahan,
               void *stream) {
    if (!rowmajor_dev(X) || !rowmajor_dev(V) || !rowmajor_dev(W)) return SP_ERR_ARG;
    if (V->nrows != W->nrows || X->nrows != V->ncols || X->ncols != W->ncols) return SP_ERR_DIM;
    if (V->dtype != W->dtype || X->dtype != V->dtype || (V->dtype != SP_F64 && V->dtype != SP_F32))
        return SP_ERR_DTYPE;
    const int m = V->ncols, k = W->ncols;
    if (m < 1 || k < 1) return SP_ERR_ARG;
    if (m > sp::kTsmMax || k > sp::kTsmMax) return SP_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = V->nrows;
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>(sp::sms_blocks(4), (n + sp::kTileRows - 1) / sp::kTileRows));
    const int64_t rpb = std::max<int64_t>(sp::kTileRows,
                                          ((n + nb - 1) / nb + sp::kTileRows - 1) / sp::kTileRows * sp::kTileRows);
    nb = (int)std::max<int64_t>(1, (n + rpb - 1) / rpb);
    DevBufPtr part;
    SP_TRY(sp::dev_alloc(part, (size_t)nb * m * k * sizeof(double), s));
    const int fin = (m * k + 255) / 256;
#define SP_TSM_LAUNCH(T, KH)                                                                                       \
    sp::k_tsmttsm_part<T, KH><<<nb, sp::kTsmThreads, 0, s>>>((const T *)V->ptr, V->ld, (const T *)W->ptr, W->ld, n, \
                                                             m, k, rpb, (double *)part->ptr);                         \
    sp::k_tsmttsm_final<T, KH><<<fin, 256, 0, s>>>((const double *)part->ptr, nb, m, k, alpha, beta, (T *)X->ptr,   \
                                                   X->ld);
    if (V->dtype == SP_F64) {
        if (kahan) {
            SP_TSM_LAUNCH(double, true)
        } else {
            SP_TSM_LAUNCH(double, false)
        }
    } else {
        if (kahan) {
            SP_TSM_LAUNCH(float, true)
        } else {
            SP_TSM_LAUNCH(float, false)
        }
    }
#undef SP_TSM_LAUNCH
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}

int sp_tsmm(sp_dense *W, const sp_dense *V, const sp_dense *X, double alpha, double beta, void *stream) {
    if (!rowmajor_dev(X) || !rowmajor_dev(V) || !rowmajor_dev(W)) return SP_ERR_ARG;
    if (V->nrows != W->nrows || X->nrows != V->ncols || X->ncols != W->ncols) return SP_ERR_DIM;
    if (V->dtype != W->dtype || X->dtype != V->dtype || (V->dtype != SP_F64 && V->dtype != SP_F32))
        return SP_ERR_DTYPE;
    const int m = V->ncols, k = W->ncols;
    if (m < 1 || k < 1) return SP_ERR_ARG;
    if (m > sp::kTsmMax || k > sp::kTsmMax) return SP_ERR_UNSUPPORTED;
    const bool inplace = W->ptr == V->ptr;
    if (inplace && (W->ld != V->ld || m != k)) return SP_ERR_ARG;
    // a partial overlap of W with V or X (other than the in-place form) is refused
    const size_t xs = V->dtype == SP_F64 ? 8 : 4;
    auto span = [&](const sp_dense *d) { return (size_t)d->ld * d->nrows * xs; };
    auto overl = [&](const sp_dense *a, const sp_dense *b) {
        const char *pa = (const char *)a->ptr, *pb = (const char *)b->ptr;
        return pa < pb + span(b) && pb < pa + span(a);
    };
    if ((!inplace && overl(W, V)) || overl(W, X)) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = V->nrows;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(sp::sms_blocks(8), (n + sp::kTileRows - 1) / sp::kTileRows));
    if (V->dtype == SP_F64)
        sp::k_tsmm<double><<<nb, sp::kTsmThreads, 0, s>>>((const double *)V->ptr, V->ld, (const double *)X->ptr, X->ld,
                                                          (double *)W->ptr, W->ld, n, m, k, alpha, beta);
    else
        sp::k_tsmm<float><<<nb, sp::kTsmThreads, 0, s>>>((const float *)V->ptr, V->ld, (const float *)X->ptr, X->ld,
                                                         (float *)W->ptr, W->ld, n, m, k, (float)alpha, (float)beta);
    SP_CUDA(cudaGetLastError());
    return SP_OK;
}
