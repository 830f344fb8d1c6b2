// kernels_solve.cu -- the B-step of an altGDmin iteration (Alg. 2): for each
// frame k the r x r least squares  G_k b_k = h_k  with
//   G_k = (A_k U)^H (A_k U) = sum over the frame's sampled rows ky and the
//         coils j of the row Grams P[j][ky] (k_fwd_rows),
//   h_k = (A_k U)^H y_k = U^H Z[:, k] (totals left by k_gdqr),
// solved by an FP32 Cholesky factorisation, one block per frame.
#include <math.h>

#include "common.cuh"
#include "internal.h"

#define RMAXC 16   // compile-time bound on the rank
#define NT 256     // threads per block

__global__ void __launch_bounds__(NT) k_solve(const float2 *__restrict__ Ppart, const double2 *__restrict__ htot,
                                              const int32_t *__restrict__ lineptr,
                                              const int32_t *__restrict__ framerows, int ny, int r, int ncg,
                                              float2 *__restrict__ B, unsigned int *status) {
    __shared__ double sP[RMAXC * (RMAXC + 1)];
    __shared__ float2 sG[RMAXC * RMAXC];
    __shared__ float sinv[RMAXC];
    __shared__ int s_rows[256];
    const int k = blockIdx.x;
    const int np = r * (r + 1) / 2, rr = r * r;
    const int lp = lineptr[k], L = lineptr[k + 1] - lp;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s_rows[i] = framerows[lp + i];
    __syncthreads();
    // G_k pairs: sum over the frame's (row, coil) items of the row Grams
    block_sum(np, L * ncg, sP, [=](int p, int it) {
        const int i = it / ncg, g = it - i * ncg;
        return __ldg(Ppart + ((size_t)g * ny + s_rows[i]) * np + p);
    });
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        const int p = a <= b ? pair_index(a, b, r) : pair_index(b, a, r);
        sG[e] = make_float2((float)sP[2 * p], (float)(a <= b ? sP[2 * p + 1] : -sP[2 * p + 1]));
    }
    __syncthreads();
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    const bool ok = (L > 0) && warp_chol32<RMAXC>(sG, r, sinv);
    float2 h = make_float2(0.f, 0.f);
    if (lane < r) {
        const double2 v = __ldcg(htot + rr + (size_t)k * r + lane);
        h = make_float2((float)v.x, (float)v.y);
    }
    float2 x = make_float2(0.f, 0.f);
    if (ok) x = warp_chol_solve32(sG, sinv, r, h);
    if (!ok && lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_LS);
    if (lane < r) B[(size_t)k * r + lane] = x;
}

cudaError_t launch_solve(lrccs_ctx *c) {
    prof_begin(c, KID_SOLVE);
    k_solve<<<c->q, NT, 0, c->stream>>>(c->d_P, c->d_tot, c->d_lineptr, c->d_framerows, c->ny, c->r, c->ncg,
                                        c->d_B, c->d_status);
    prof_end(c, KID_SOLVE);
    return cudaGetLastError();
}
