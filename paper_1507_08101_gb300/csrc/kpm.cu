// Chebyshev moments of the kernel polynomial method on the augmented product.
//
// Sec. "Kernel fusion" names the kernel polynomial method as the solver the
// fused SpMMV serves.  With A~ = (A - b I) / a and w_0 = x, the Chebyshev
// recurrence w_1 = A~ w_0, w_{n+1} = 2 A~ w_n - w_{n-1} is one augmented
// product per step (alpha = 2/a, gamma = b, beta = -1, y holding w_{n-1} on
// entry), and its fused <y,y> and <x,y> give two moments per step by the
// product rules of the Chebyshev polynomials (A. Weisse et al., "The kernel
// polynomial method", Rev. Mod. Phys. 78 (2006)):
//     mu_{2n}   = 2 <w_n, w_n>     - mu_0
//     mu_{2n+1} = 2 <w_{n+1}, w_n> - mu_1
// Step 0 (w_1 = A~ w_0) also yields mu_0 = <w_0, w_0> (the fused <x,x>) and
// mu_1 = <w_0, w_1>.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sp {

// mu[k * w + c] from the per-step dots d[n][q * w + c] (q: 0 yy, 1 xy, 2 xx)
__global__ void k_kpm_assemble(const double *__restrict__ d, int w, int nmom, double *__restrict__ mu) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nmom * w; t += gridDim.x * blockDim.x) {
        const int k = t / w, c = t - k * w;
        const double mu0 = d[2 * w + c], mu1 = d[w + c];
        double v;
        if (k == 0) {
            v = mu0;
        } else if (k == 1) {
            v = mu1;
        } else if ((k & 1) == 0) {
            const int n = k / 2;  // <w_n, w_n> is the <y,y> of step n - 1
            v = __fma_rn(2.0, d[(int64_t)(n - 1) * 3 * w + c], -mu0);
        } else {
            const int n = k / 2;  // <w_{n+1}, w_n> is the <x,y> of step n
            v = __fma_rn(2.0, d[(int64_t)n * 3 * w + w + c], -mu1);
        }
        mu[t] = v;
    }
}

}  // namespace sp

int sp_kpm_moments(const sp_mat *A, const sp_dense *x, int32_t nmom, double a, double b, double *mu, void *stream) {
    if (sp::dense_scattered(x)) return sp::scattered_refused("sp_kpm_moments");
    if (!A || !x || !mu || nmom < 1) return SP_ERR_ARG;
    if (!(a != 0.0) || !std::isfinite(a) || !std::isfinite(b)) return SP_ERR_ARG;
    const sp::Pattern &P = *A->pat;
    if (P.nrows != P.ncols || x->nrows != P.nrows) return SP_ERR_DIM;
    if (x->layout != SP_ROW_MAJOR) return SP_ERR_ARG;
    const int w = x->ncols;
    if (w < 1) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // steps: step 0 gives mu_0..mu_2, step n >= 1 gives mu_{2n+1}, mu_{2n+2}
    const int K = nmom - 1;
    const int nsteps = 1 + std::max(0, (K - 2 + 1) / 2);
    // working memory is stream-ordered, so a call does not synchronise the device
    const size_t xs = x->dtype == SP_F64 ? 8 : 4;
    sp::Tmp ub(s), vb(s), dots(s), dmu(s);
    int rc = ub.alloc((size_t)P.nrows * w * xs);
    if (rc == SP_OK) rc = vb.alloc((size_t)P.nrows * w * xs);
    if (rc == SP_OK) rc = dots.alloc((size_t)nsteps * 3 * w * sizeof(double));
    if (rc == SP_OK) rc = dmu.alloc((size_t)nmom * w * sizeof(double));
    sp_dense *u = nullptr, *v = nullptr;
    if (rc == SP_OK) rc = sp_dense_view(&u, ub.p, P.nrows, w, w, x->dtype, SP_ROW_MAJOR);
    if (rc == SP_OK) rc = sp_dense_view(&v, vb.p, P.nrows, w, w, x->dtype, SP_ROW_MAJOR);
    if (rc == SP_OK) {
        cudaError_t e = cudaMemcpy2DAsync(u->ptr, (size_t)w * xs, x->ptr, (size_t)x->ld * xs, (size_t)w * xs,
                                          (size_t)P.nrows, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            sp_internal_note_cuda_error(e, "kpm copy of x", __FILE__, __LINE__);
            rc = SP_ERR_CUDA;
        }
    }
    double *d = rc == SP_OK ? dots.as<double>() : nullptr;
    const double gamma = b;
    for (int n = 0; n < nsteps && rc == SP_OK; ++n) {
        sp_spmv_opts o = SP_SPMV_OPTS_INIT;
        o.gamma = &gamma;
        o.dot = d + (size_t)n * 3 * w;
        if (n == 0) {
            // v = w_1 = A~ w_0, with <w_0,w_0>, <w_0,w_1>, <w_1,w_1>
            o.flags = SP_SPMV_SCALE | SP_SPMV_SHIFT | SP_SPMV_DOT_YY | SP_SPMV_DOT_XY | SP_SPMV_DOT_XX;
            o.alpha = 1.0 / a;
            rc = sp_spmv(v, A, u, &o, stream);
        } else {
            // u = w_{n+1} = 2 A~ w_n - w_{n-1} (u holds w_{n-1}, v holds w_n)
            o.flags = SP_SPMV_SCALE | SP_SPMV_SHIFT | SP_SPMV_AXPBY | SP_SPMV_DOT_YY | SP_SPMV_DOT_XY;
            o.alpha = 2.0 / a;
            o.beta = -1.0;
            rc = sp_spmv(u, A, v, &o, stream);
            std::swap(u, v);
        }
    }
    if (rc == SP_OK) {
        const int threads = 256, blocks = std::max(1, std::min(1024, (nmom * w + threads - 1) / threads));
        sp::k_kpm_assemble<<<blocks, threads, 0, s>>>(d, w, nmom, dmu.as<double>());
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(mu, dmu.p, (size_t)nmom * w * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            sp_internal_note_cuda_error(e, "kpm moments", __FILE__, __LINE__);
            rc = SP_ERR_CUDA;
        }
    } else {
        cudaStreamSynchronize(s);
    }
    if (u) sp_dense_destroy(u, stream);  // views: the memory goes back with ub, vb
    if (v) sp_dense_destroy(v, stream);
    return rc;
}
