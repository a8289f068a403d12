// a0. Response spectrum (Sec. III-A-2: the per-impact response spectra are computed once;
// Eq. interlaced: R[j, k] = i[j, -k]).
//
// For the kept impact j of each channel pair and every padded frequency
// (ky, kx, f) of the 16 x 16 x lt grid:
//   Rhat[j](ky, kx, f) = 1/(16*16*lt) sum_{K, tau} i[K][j][tau]
//                          exp(+2 pi i (Ky ky + Kx kx) / 16) exp(-2 pi i tau f / lt)
// (the spatial sign is + because R[j, k] = i[j, -k]; the 1/N of the inverse FFT
// is folded in).  Evaluated once per response as two direct DFT stages in FP64
// with exact twiddle arguments, rounded to complex64, and stored as
//   rhat[k1][pair][k2][rhat_kk(ky, kx)]   with f = k1 + G2 k2, G2 = lt / 32,
// so that the convolution CTA owning the 32 bins of class k1 streams one
// contiguous 64 KB slab per channel pair.
#include <cmath>
#include <vector>

#include "tred_internal.cuh"

namespace tred {

// Stage 1: T[pair][Ky][Kx][f] = sum_tau i[Ky][Kx][j][tau] W_lt^{tau f} (FP64).
__global__ void k_resp_time(const float *__restrict__ resp, const int32_t *__restrict__ pair_j,
                            int npairs, int kp, int ns, int nr, int lt,
                            const double2 *__restrict__ wlt, double2 *__restrict__ T) {
    const int64_t total = (int64_t)npairs * kp * kp * lt;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(idx % lt);
        int64_t r = idx / lt;
        const int Kx = (int)(r % kp);
        r /= kp;
        const int Ky = (int)(r % kp);
        const int p = (int)(r / kp);
        const int j = pair_j[2 * p];
        const int jy = j / ns, jx = j % ns;
        const float *ir = resp + ((((int64_t)Ky * kp + Kx) * ns + jy) * ns + jx) * nr;
        double re = 0.0, im = 0.0;
        for (int tau = 0; tau < nr; ++tau) {
            const double v = (double)ir[tau];
            const double2 w = wlt[((int64_t)tau * f) % lt];
            re = fma(v, w.x, re);
            im = fma(v, w.y, im);
        }
        T[idx] = make_double2(re, im);
    }
}

// Stage 2: spatial DFT with the + sign, scaling, layout change to the conv order.
__global__ void k_resp_space(const double2 *__restrict__ T, int npairs, int kp, int lt, int G2,
                             const double2 *__restrict__ w16, double scale,
                             float2 *__restrict__ rhat) {
    const int R = (kp - 1) / 2;
    const int64_t total = (int64_t)npairs * lt * LP * LP;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(idx % LP);
        int64_t r = idx / LP;
        const int ky = (int)(r % LP);
        r /= LP;
        const int f = (int)(r % lt);
        const int p = (int)(r / lt);
        double re = 0.0, im = 0.0;
        for (int Ky = 0; Ky < kp; ++Ky)
            for (int Kx = 0; Kx < kp; ++Kx) {
                const double2 t = T[(((int64_t)p * kp + Ky) * kp + Kx) * lt + f];
                // exp(+2 pi i m / 16) = conj(W16^m), m = (Ky - R) ky + (Kx - R) kx
                int m = ((Ky - R) * ky + (Kx - R) * kx) % LP;
                if (m < 0) m += LP;
                const double2 w = w16[m];
                const double wr = w.x, wi = -w.y;
                re += t.x * wr - t.y * wi;
                im += t.x * wi + t.y * wr;
            }
        rhat[rhat_bin(f, p, npairs, G2) + rhat_kk(ky, kx)] =
            make_float2((float)(re * scale), (float)(im * scale));
    }
}

int launch_response(tred_handle *h, const float *resp, cudaStream_t s) {
    const int kp = h->g.kp, ns = h->g.n_sub, nr = h->g.nr, lt = h->g.lt, G2 = lt / 32;
    const int NP = h->d.npairs;
    std::vector<double2> wlt(lt), w16(LP);
    for (int k = 0; k < lt; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)lt;
        wlt[k] = make_double2(std::cos(a), -std::sin(a));
    }
    for (int k = 0; k < LP; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)LP;
        w16[k] = make_double2(std::cos(a), -std::sin(a));
    }
    double2 *d_wlt = nullptr, *d_w16 = nullptr, *d_T = nullptr;
    const size_t nT = (size_t)NP * kp * kp * lt;
    int rc = check_cuda(h, cudaMalloc(&d_wlt, sizeof(double2) * lt), "alloc resp twiddles");
    if (!rc) rc = check_cuda(h, cudaMalloc(&d_w16, sizeof(double2) * LP), "alloc resp twiddles");
    if (!rc) rc = check_cuda(h, cudaMalloc(&d_T, sizeof(double2) * nT), "alloc resp stage");
    if (!rc) rc = check_cuda(h, cudaMemcpyAsync(d_wlt, wlt.data(), sizeof(double2) * lt, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) rc = check_cuda(h, cudaMemcpyAsync(d_w16, w16.data(), sizeof(double2) * LP, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) {
        const int grid = num_sms(h) * 8;
        k_resp_time<<<grid, 256, 0, s>>>(resp, h->pair_j, NP, kp, ns, nr, lt, d_wlt, d_T);
        const double scale = 1.0 / ((double)LP * LP * lt);
        k_resp_space<<<grid, 256, 0, s>>>(d_T, NP, kp, lt, G2, d_w16, scale, h->rhat);
        h->launches += 2;
        rc = check_cuda(h, cudaGetLastError(), "response launch");
    }
    // the staging buffers are freed after the stream drains (set-up path, once)
    cudaError_t e = cudaStreamSynchronize(s);
    if (!rc) rc = check_cuda(h, e, "response sync");
    cudaFree(d_wlt);
    cudaFree(d_w16);
    cudaFree(d_T);
    return rc;
}

}  // namespace tred
