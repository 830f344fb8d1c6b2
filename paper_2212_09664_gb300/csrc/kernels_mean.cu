// kernels_mean.cu -- the mean step of Alg. 1 on sm_103a:
//   step 1   zbar = argmin_z sum_k ||y_k - A_k z||^2, by conjugate gradients on
//            the normal equations A^H A z = A^H y (CGLS) from z = 0;
//   step 2a  y~_k = y_k - A_k zbar.
// The normal operator A^H A = sum_k A_k^H A_k is the iteration's transform
// pipeline at rank 1 with b_k = 1 (launch_normal_op in kernels_iter.cu): with
// line masks it is sum_j conj(d_j) o F_y^H[c_ky F_y(d_j o z)], c_ky the number
// of frames that sample row ky.  This file holds the right-hand side, one CG
// step and the residual pass.
//
// CG vectors live in the context's n x r buffers (first column): p in U (the
// operator's input), A^H A p in U+ (its output), z in U_{t-1}, s = A^H r in
// the gradient buffer.  The CG scalars are FP64, summed in a fixed order.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

#define CG_THREADS 1024

// Sum over the block of one FP64 value per thread: warp shuffles, then the
// warps in order (deterministic).  red holds 33 doubles.
static __device__ double block_sum_fp64(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();   // every thread has read red[32] of a previous call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// s = A^H y = sum_k Z[:, k] (Z = [A_k^H y_k], row-major i q + k), p = s, z = 0,
// B = 1 (q x 1); cg = {||s||^2, 0, 0}.  One block.
__global__ void __launch_bounds__(CG_THREADS) k_cg_init(const float2 *__restrict__ Z, int n, int q, float2 *s,
                                                        float2 *p, float2 *z, float2 *B, double *cg) {
    __shared__ double red[33];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        for (int k = 0; k < q; ++k) {
            const float2 a = Z[(size_t)i * q + k];
            v.x += a.x;
            v.y += a.y;
        }
        s[i] = v;
        p[i] = v;
        z[i] = make_float2(0.f, 0.f);
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int k = threadIdx.x; k < q; k += blockDim.x) B[k] = make_float2(1.f, 0.f);
    const double g = block_sum_fp64(acc, red);
    if (threadIdx.x == 0) {
        cg[0] = g;
        cg[1] = 0.0;
        cg[2] = 0.0;
    }
}

// One CG step on A^H A z = A^H y, given w = A^H A p:
//   alpha = gamma / <p, w>;  z += alpha p;  s -= alpha w;
//   gamma' = ||s||^2;  p = s + (gamma' / gamma) p.
// cg = {gamma, alpha, stop}: stop = 1 (and nothing updated) when <p, w> <= 0.
// One block; each thread updates the same entries in every pass.
__global__ void __launch_bounds__(CG_THREADS) k_cg_step(float2 *p, const float2 *__restrict__ w, float2 *z,
                                                        float2 *s, int n, double *cg) {
    __shared__ double red[33];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = p[i], b = w[i];
        acc += (double)a.x * b.x + (double)a.y * b.y;   // Re(conj(p_i) w_i)
    }
    const double dot = block_sum_fp64(acc, red);
    const double gamma = cg[0];
    if (!(dot > 0.0) || !(gamma > 0.0)) {
        if (threadIdx.x == 0) cg[2] = 1.0;
        return;
    }
    const double alpha_d = gamma / dot;
    const float alpha = (float)alpha_d;
    acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 a = p[i], b = w[i];
        float2 zz = z[i], ss = s[i];
        zz.x = fmaf(alpha, a.x, zz.x);
        zz.y = fmaf(alpha, a.y, zz.y);
        ss.x = fmaf(-alpha, b.x, ss.x);
        ss.y = fmaf(-alpha, b.y, ss.y);
        z[i] = zz;
        s[i] = ss;
        acc += (double)ss.x * ss.x + (double)ss.y * ss.y;
    }
    const double g2 = block_sum_fp64(acc, red);
    const float beta = (float)(g2 / gamma);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 ss = s[i], a = p[i];
        p[i] = make_float2(fmaf(beta, a.x, ss.x), fmaf(beta, a.y, ss.y));
    }
    if (threadIdx.x == 0) {
        cg[0] = g2;
        cg[1] = alpha_d;
    }
}

// y~ = y - A z on every sampled line.  T holds F_y(d_j o z) on the sampled rows
// (rank 1: T[(j ny + ky) nx + x]).  Row rr = j nl_k + i of frame k (coil j,
// line i, ky = framerows[lp_k + i]) is y[(C lp_k + rr) nx + kx]; the pass
// applies F_x (unitary) to T_j[ky, :] and subtracts.  Grid (ceil(C nl_max / 8), q).
template <int P>
__global__ void __launch_bounds__(256) k_mean_resid(const float2 *__restrict__ y, const float2 *__restrict__ T,
                                                     const int32_t *__restrict__ framerows,
                                                     const int32_t *__restrict__ lineptr, float2 *__restrict__ ytil,
                                                     int ny, int nc, const float2 *__restrict__ g_tw, float scale) {
    constexpr int N = 32 * P;
    constexpr int ROWS = 8, TPR = ROWS + 1;
    __shared__ float2 s_tw[N];
    __shared__ float2 tile[N * TPR];
    const int k = blockIdx.y;
    const int lp = lineptr[k], nl = lineptr[k + 1] - lp;
    const int rows_k = nc * nl;
    const int r0 = blockIdx.x * ROWS;
    if (r0 >= rows_k) return;   // the same for every thread of the block
    load_twiddles(s_tw, g_tw, N);
    for (int e = threadIdx.x; e < ROWS * N; e += blockDim.x) {
        const int row = e / N, x = e - row * N;
        const int rr = r0 + row;
        float2 a = make_float2(0.f, 0.f);
        if (rr < rows_k) {
            const int j = rr / nl, i = rr - j * nl;
            const int ky = framerows[lp + i];
            a = T[((size_t)j * ny + ky) * N + x];
        }
        tile[x * TPR + row] = a;
    }
    __syncthreads();
    fft::tile_dft<N, false>(tile, TPR, ROWS, s_tw, scale);
    for (int e = threadIdx.x; e < ROWS * N; e += blockDim.x) {
        const int row = e / N, kx = e - row * N;
        const int rr = r0 + row;
        if (rr < rows_k) {
            const size_t off = ((size_t)nc * lp + rr) * N + kx;
            const float2 a = y[off], b = tile[kx * TPR + row];
            ytil[off] = make_float2(a.x - b.x, a.y - b.y);
        }
    }
}

#define DISPATCH_P(PV, ...)                                           \
    switch (PV) {                                                      \
        case 1: { constexpr int P_ = 1; __VA_ARGS__; } break;                 \
        case 2: { constexpr int P_ = 2; __VA_ARGS__; } break;                 \
        case 3: { constexpr int P_ = 3; __VA_ARGS__; } break;                 \
        case 4: { constexpr int P_ = 4; __VA_ARGS__; } break;                 \
        case 5: { constexpr int P_ = 5; __VA_ARGS__; } break;                 \
        case 6: { constexpr int P_ = 6; __VA_ARGS__; } break;                 \
        case 7: { constexpr int P_ = 7; __VA_ARGS__; } break;                 \
        case 8: { constexpr int P_ = 8; __VA_ARGS__; } break;                 \
        default: return cudaErrorInvalidValue;                         \
    }

cudaError_t launch_cg_init(lrccs_ctx *c, double *cg) {
    prof_begin(c, KID_CG_INIT);
    k_cg_init<<<1, CG_THREADS, 0, c->stream>>>(c->d_Z, c->n, c->q, c->d_G, c->d_U, c->d_Uprev, c->d_B, cg);
    prof_end(c, KID_CG_INIT);
    return cudaGetLastError();
}

cudaError_t launch_cg_step(lrccs_ctx *c, double *cg) {
    prof_begin(c, KID_CG_STEP);
    k_cg_step<<<1, CG_THREADS, 0, c->stream>>>(c->d_U, c->d_Up, c->d_Uprev, c->d_G, c->n, cg);
    prof_end(c, KID_CG_STEP);
    return cudaGetLastError();
}

cudaError_t launch_mean_resid(lrccs_ctx *c, const float2 *d_y, float2 *d_ytil, int nl_max) {
    if (nl_max < 1) return cudaSuccess;
    const float sx = (float)(1.0 / sqrt((double)c->nx));
    const dim3 grid((unsigned)((c->nc * nl_max + 7) / 8), (unsigned)c->q);
    DISPATCH_P(c->px, {
        prof_begin(c, KID_MEAN_RESID);
        k_mean_resid<P_><<<grid, 256, 0, c->stream>>>(d_y, c->d_T, c->d_framerows, c->d_lineptr, d_ytil, c->ny,
                                                      c->nc, c->d_twx, sx);
        prof_end(c, KID_MEAN_RESID);
    });
    return cudaGetLastError();
}
