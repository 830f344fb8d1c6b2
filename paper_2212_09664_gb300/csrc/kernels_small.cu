// kernels_small.cu -- the r x r parts of an altGDmin iteration (Alg. 2):
// the per-frame least squares of the B-step (FP64 Cholesky of G_k) and the
// GD step with CholeskyQR2 re-orthonormalisation (FP64 Cholesky of the r x r
// Grams), with every grid reduction finished by the last block to arrive.
//
// The pixel-parallel kernels stage their whole pixel range (or large chunks
// of it) with one batch of cp.async copies, so a block waits for global
// memory once per chunk instead of once per element.
#include <math.h>

#include "common.cuh"
#include "internal.h"

#define RMAXC 16   // compile-time bound on the rank
#define NT 256     // threads per block of the pixel-parallel kernels

// Expand packed upper-triangle pairs (FP64 re, im) into a full Hermitian matrix.
static __device__ void expand_pairs(const double *packed, int r, double *A) {
    const int np = r * (r + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        int a, b;
        pair_of(p, r, a, b);
        const double re = packed[2 * p], im = packed[2 * p + 1];
        A[(a * r + b) * 2] = re;
        A[(a * r + b) * 2 + 1] = im;
        A[(b * r + a) * 2] = re;
        A[(b * r + a) * 2 + 1] = -im;
    }
    __syncthreads();
}

// Stage count float2 from global src to shared dst (cp.async, 16 B when aligned).
static __device__ void stage(float2 *dst, const float2 *src, int count) {
    if (((((uintptr_t)src) | smem_u32(dst)) & 15) == 0 && (count & 1) == 0) {
        for (int e = threadIdx.x; e < count / 2; e += blockDim.x) cp_async16(dst + 2 * e, src + 2 * e);
    } else {
        for (int e = threadIdx.x; e < count; e += blockDim.x) cp_async8(dst + e, src + e);
    }
}

// Hermitian Gram partial sum_i conj(u_i[a]) u_i[b] over cn rows of s_u
// (row length r), spread over all threads: thread = (pair p, pixel group g).
// Returns the block's sum for pair threadIdx.x (< np) via s_red.
static __device__ float2 gram_partial(const float2 *s_u, int cn, int r, float2 *s_red) {
    const int np = r * (r + 1) / 2;
    const int KG = max(1, (int)blockDim.x / np);
    const int p = threadIdx.x % np, g = threadIdx.x / np;
    float2 acc = make_float2(0.f, 0.f);
    if (g < KG) {
        int a, b;
        pair_of(p, r, a, b);
        for (int ii = g; ii < cn; ii += KG) cfmac(acc, s_u[ii * r + a], s_u[ii * r + b]);
        s_red[g * np + p] = acc;
    }
    __syncthreads();
    float2 s = make_float2(0.f, 0.f);
    if (threadIdx.x < np)
        for (int gg = 0; gg < KG; ++gg) s = cadd(s, s_red[gg * np + threadIdx.x]);
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------- C: per-frame LS
// G_k b_k = h_k with G_k = (A_k U)^H (A_k U) = sum over the frame's sampled
// rows and the coils of the row Grams P, and h_k = U^H Z[:, k] (Alg. 2, B-update).

__global__ void __launch_bounds__(NT) k_solve(const float2 *__restrict__ Ppart, const float2 *__restrict__ Hpart,
                                              const int32_t *__restrict__ lineptr,
                                              const int32_t *__restrict__ framerows, int ny, int r, int q, int ncg,
                                              int nblkH, float2 *__restrict__ B, unsigned int *status) {
    __shared__ double sP[RMAXC * (RMAXC + 1)];
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sh[RMAXC * 2];
    __shared__ double sx[RMAXC * 2];
    __shared__ double sinv[RMAXC];
    __shared__ int s_rows[256];
    const int k = blockIdx.x;
    const int np = r * (r + 1) / 2;
    const int lp = lineptr[k], L = lineptr[k + 1] - lp;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s_rows[i] = framerows[lp + i];
    __syncthreads();
    // G_k pairs: sum over the frame's (row, coil) items of the row Grams
    block_sum(np, L * ncg, sP, [=](int p, int it) {
        const int i = it / ncg, g = it - i * ncg;
        return __ldg(Ppart + ((size_t)g * ny + s_rows[i]) * np + p);
    });
    // h_k = U^H Z[:, k] from the per-block partials of the previous H kernel
    block_sum(r, nblkH, sh, [=](int l, int blk) { return __ldcg(Hpart + ((size_t)blk * q + k) * r + l); });
    expand_pairs(sP, r, sG);
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    const bool ok = (L > 0) && warp_cholesky_rl(sG, r, sinv);
    if (ok) warp_chol_solve_rl(sG, sinv, r, sh, sx);
    if (!ok && lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_LS);
    for (int l = lane; l < r; l += 32)
        B[(size_t)k * r + l] = ok ? make_float2((float)sx[2 * l], (float)sx[2 * l + 1]) : make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------- F, G, H: GD step and CholeskyQR2
// Each block owns pixels [i0, i1); chunk = pixels staged at once (host-chosen
// so that the staging fits shared memory).

// F: U+ = U - eta grad (or U+ as given, at init), the Gram of U+, and in the
// last block R1^{-1} with U+^H U+ = R1^H R1.
__global__ void __launch_bounds__(NT) k_gd_gram(const float2 *__restrict__ U, const float2 *__restrict__ Gr,
                                                 float2 *__restrict__ Up, const double *__restrict__ scal,
                                                 float2 *gpart, unsigned int *counter, double *R1,
                                                 unsigned int *status, int n, int r, int chunk, int from_grad) {
    extern __shared__ __align__(16) float2 smem[];
    float2 *s_u = smem;                     // chunk * r
    float2 *s_g = s_u + chunk * r;          // chunk * r
    __shared__ float2 s_red[NT];
    __shared__ double sP[RMAXC * (RMAXC + 1)];
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sLi[RMAXC * RMAXC * 2];
    const int np = r * (r + 1) / 2;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const float eta = from_grad ? (float)scal[SC_ETA] : 0.f;
    float2 tot = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        if (from_grad) {
            stage(s_u, U + (size_t)c0 * r, cn * r);
            stage(s_g, Gr + (size_t)c0 * r, cn * r);
        } else {
            stage(s_u, Up + (size_t)c0 * r, cn * r);
        }
        cp_async_commit();
        cp_async_wait();
        __syncthreads();
        if (from_grad) {
            for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
                const float2 v = csub(s_u[e], cscale(s_g[e], eta));
                s_u[e] = v;
                Up[(size_t)c0 * r + e] = v;
            }
            __syncthreads();
        }
        tot = cadd(tot, gram_partial(s_u, cn, r, s_red));
    }
    if (threadIdx.x < np) gpart[(size_t)blockIdx.x * np + threadIdx.x] = tot;
    if (!last_block_arrive(counter)) return;
    block_reduce_rows(gpart, gridDim.x, np, sP);
    expand_pairs(sP, r, sG);
    if ((threadIdx.x >> 5) != 0) return;
    // U+^H U+ = L L^H (FP64); R1 = L^H is handed on as L and 1/diag in FP32
    float2 *Lf = (float2 *)R1;
    float *invf = (float *)(Lf + r * r);
    const int lane = threadIdx.x & 31;
    const bool ok = warp_cholesky_rl(sG, r, sLi);
    if (!ok && lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_QR);
    for (int e = lane; e < r * r; e += 32) {
        const int a = e / r, b = e - a * r;
        Lf[e] = ok ? (b <= a ? make_float2((float)sG[2 * e], (float)sG[2 * e + 1]) : make_float2(0.f, 0.f))
                   : make_float2(a == b ? 1.f : 0.f, 0.f);
    }
    for (int a = lane; a < r; a += 32) invf[a] = ok ? (float)sLi[a] : 1.f;
}

// Store the FP64 factor L (lower, in A) of R1 = L^H as FP32 L and 1/diag for
// the pixel kernels (or the identity when the factorisation failed).
static __device__ void store_r1(const double *A, const double *invd, bool ok, int r, double *R1) {
    float2 *Lf = (float2 *)R1;
    float *invf = (float *)(Lf + r * r);
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < r * r; e += 32) {
        const int a = e / r, b = e - a * r;
        Lf[e] = ok ? (b <= a ? make_float2((float)A[2 * e], (float)A[2 * e + 1]) : make_float2(0.f, 0.f))
                   : make_float2(a == b ? 1.f : 0.f, 0.f);
    }
    for (int a = lane; a < r; a += 32) invf[a] = ok ? (float)invd[a] : 1.f;
}

// F: the gradient of Alg. 2, grad = Gk - Z B^H (Gk = sum_j conj(d_j) F^H K_j
// from k_adj_cols), and partial sums of grad^H grad, U^H grad and U^H U.  The
// last block sets eta = eta_c / ||grad||_2 at t = 1, forms
//     G1 = (U - eta grad)^H (U - eta grad) = U^H U - eta (U^H grad + grad^H U) + eta^2 grad^H grad
// in FP64 and factors it (FP64 Cholesky) into R1 for CholeskyQR2.
#define GSLOT 3   // partial-sum entries per thread: 2 np + r^2 <= 256 * 3
__global__ void __launch_bounds__(NT) k_grad(const float2 *__restrict__ Gk, const float2 *__restrict__ Z,
                                              const float2 *__restrict__ B, const float2 *__restrict__ U,
                                              float2 *__restrict__ Gr, double *scal, float2 *gpart,
                                              unsigned int *counter, double *R1, unsigned int *status, int n, int r,
                                              int q, int chunk, double eta_c) {
    extern __shared__ __align__(16) float2 smem[];
    float2 *s_g = smem;                   // chunk * r
    float2 *s_u = s_g + chunk * r;        // chunk * r
    float2 *s_z = s_u + chunk * r;        // chunk * q
    __shared__ float2 sB[128 * RMAXC];
    __shared__ double sAll[(2 * RMAXC * (RMAXC + 1) / 2 + RMAXC * RMAXC) * 2];
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sInv[RMAXC];
    __shared__ float2 sA[RMAXC * RMAXC];
    __shared__ float s_c[16], s_s[16];
    __shared__ float2 s_e[16];
    __shared__ int s_cnt;
    __shared__ double s_eta;
    const int np = r * (r + 1) / 2, rr = r * r;
    const int len = 2 * np + rr;          // [grad^H grad pairs | U^H grad | U^H U pairs]
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int e = threadIdx.x; e < q * r; e += blockDim.x) sB[e] = B[e];
    int sa[GSLOT], sb[GSLOT], kind[GSLOT];
#pragma unroll
    for (int u = 0; u < GSLOT; ++u) {
        const int e = threadIdx.x + NT * u;
        kind[u] = -1;
        sa[u] = sb[u] = 0;
        if (e < np) { kind[u] = 0; pair_of(e, r, sa[u], sb[u]); }
        else if (e < np + rr) { kind[u] = 1; sa[u] = (e - np) / r; sb[u] = (e - np) - sa[u] * r; }
        else if (e < len) { kind[u] = 2; pair_of(e - np - rr, r, sa[u], sb[u]); }
    }
    float2 acc[GSLOT];
#pragma unroll
    for (int u = 0; u < GSLOT; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        __syncthreads();
        stage(s_g, Gk + (size_t)c0 * r, cn * r);
        stage(s_u, U + (size_t)c0 * r, cn * r);
        stage(s_z, Z + (size_t)c0 * q, cn * q);
        cp_async_commit();
        cp_async_wait();
        __syncthreads();
        for (int ii = threadIdx.x; ii < cn; ii += blockDim.x) {
            float2 g[RMAXC];
#pragma unroll
            for (int l = 0; l < RMAXC; ++l) g[l] = (l < r) ? s_g[ii * r + l] : make_float2(0.f, 0.f);
            const float2 *zr = s_z + ii * q;
            for (int k = 0; k < q; ++k) {
                const float2 zk = zr[k];
#pragma unroll
                for (int l = 0; l < RMAXC; ++l)
                    if (l < r) {  // g -= zk conj(b_k[l])
                        const float2 b = sB[k * r + l];
                        g[l].x -= zk.x * b.x + zk.y * b.y;
                        g[l].y -= zk.y * b.x - zk.x * b.y;
                    }
            }
#pragma unroll
            for (int l = 0; l < RMAXC; ++l)
                if (l < r) {
                    s_g[ii * r + l] = g[l];
                    Gr[(size_t)(c0 + ii) * r + l] = g[l];
                }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < GSLOT; ++u) {
            if (kind[u] < 0) continue;
            const float2 *X = kind[u] == 0 ? s_g : s_u;   // conj(X[a]) Y[b]
            const float2 *Y = kind[u] == 2 ? s_u : s_g;
            const int a = sa[u], b = sb[u];
            for (int ii = 0; ii < cn; ++ii) cfmac(acc[u], X[ii * r + a], Y[ii * r + b]);
        }
    }
#pragma unroll
    for (int u = 0; u < GSLOT; ++u)
        if (kind[u] >= 0) gpart[(size_t)blockIdx.x * len + threadIdx.x + NT * u] = acc[u];
    if (!last_block_arrive(counter)) return;
    block_reduce_rows(gpart, gridDim.x, len, sAll);
    const double *A1 = sAll, *A2 = sAll + 2 * np, *A3 = sAll + 2 * (np + rr);
    if (threadIdx.x == 0) s_eta = scal[SC_ETA];
    if (scal[SC_ETASET] == 0.0) {
        // ||grad||_2 = sqrt(lambda_max(grad^H grad)); eta = eta_c / ||grad||_2 (Alg. 2, t = 1)
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            int a, b;
            pair_of(p, r, a, b);
            sA[a * r + b] = make_float2((float)A1[2 * p], (float)A1[2 * p + 1]);
            sA[b * r + a] = make_float2((float)A1[2 * p], (float)-A1[2 * p + 1]);
        }
        __syncthreads();
        block_jacobi(sA, r, r, nullptr, 0, s_c, s_s, s_e, &s_cnt, 30);
        if (threadIdx.x == 0) {
            float lmax = 0.f;
            for (int a = 0; a < r; ++a) lmax = fmaxf(lmax, sA[a * r + a].x);
            const double gn = sqrt((double)lmax);
            const double eta = gn > 0.0 ? eta_c / gn : 0.0;
            scal[SC_GNORM] = gn;
            scal[SC_ETA] = eta;
            scal[SC_ETASET] = 1.0;
            s_eta = eta;
        }
    }
    __syncthreads();
    const double eta = s_eta;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        const int pab = a <= b ? pair_index(a, b, r) : pair_index(b, a, r);
        const double sgn = a <= b ? 1.0 : -1.0;   // lower half: conjugate of the stored pair
        const double g1r = A1[2 * pab], g1i = sgn * A1[2 * pab + 1];
        const double g3r = A3[2 * pab], g3i = sgn * A3[2 * pab + 1];
        const double x2r = A2[2 * (a * r + b)] + A2[2 * (b * r + a)];
        const double x2i = A2[2 * (a * r + b) + 1] - A2[2 * (b * r + a) + 1];
        sG[2 * e] = g3r - eta * x2r + eta * eta * g1r;
        sG[2 * e + 1] = g3i - eta * x2i + eta * eta * g1i;
    }
    __syncthreads();
    if ((threadIdx.x >> 5) != 0) return;
    const bool ok = warp_cholesky_rl(sG, r, sInv);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, (unsigned)ST_NOT_SPD_QR);
    store_r1(sG, sInv, ok, r, R1);
}

// u1 = u+ R1^{-1} for one row, R1 = L^H: forward substitution in FP32
// (R1 has eigenvalues in [1, 1.02] here, so the solve is well conditioned).
static __device__ void tri_solve_row(const float2 *up, float2 (&u1)[RMAXC], const float2 *L, const float *invd,
                                     int r) {
#pragma unroll
    for (int b = 0; b < RMAXC; ++b) {
        if (b < r) {
            float2 v = up[b];
#pragma unroll
            for (int a = 0; a < RMAXC; ++a) {
                if (a < b) {  // v -= u1[a] conj(L[b][a])
                    const float2 l = L[b * r + a];
                    v.x -= u1[a].x * l.x + u1[a].y * l.y;
                    v.y -= u1[a].y * l.x - u1[a].x * l.y;
                }
            }
            u1[b] = cscale(v, invd[b]);
        }
    }
}

// G: the Gram of U1 = U+ R1^{-1}; in the last block the second factor of
// CholeskyQR2, M2 = R2^{-1} with U1^H U1 = R2^H R2.  U1^H U1 = I + D with
// ||D|| at FP32 rounding level, so R2 = I + up(D) + O(||D||^2), up(D) = the
// strict upper triangle of D plus half its diagonal, and R2^{-1} = I - up(D)
// to FP64 accuracy; when max |D_ab| > 1e-6 the full FP64 factorisation is used.
__global__ void __launch_bounds__(NT) k_rinv_gram(const float2 *__restrict__ U, const float2 *__restrict__ Gr,
                                                   const float2 *__restrict__ Up, const double *__restrict__ scal,
                                                   const double *__restrict__ R1,
                                                   float2 *gpart, unsigned int *counter, float2 *M,
                                                   unsigned int *status, int n, int r, int chunk, int from_grad) {
    extern __shared__ __align__(16) float2 smem[];
    float2 *s_p = smem;                     // chunk * r  (U+)
    float2 *s_u = s_p + chunk * r;          // chunk * r  (U1)
    __shared__ float2 sL[RMAXC * RMAXC];
    __shared__ float sinv[RMAXC];
    __shared__ float2 s_red[NT];
    __shared__ double sP[RMAXC * (RMAXC + 1)];
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sD[RMAXC];
    __shared__ double sX[RMAXC * RMAXC * 2];
    const int np = r * (r + 1) / 2;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const float2 *Lf = (const float2 *)R1;
    const float *invf = (const float *)(Lf + r * r);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sL[e] = Lf[e];
    for (int e = threadIdx.x; e < r; e += blockDim.x) sinv[e] = invf[e];
    const float eta = from_grad ? (float)scal[SC_ETA] : 0.f;
    float2 tot = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        __syncthreads();
        if (from_grad) {          // U+ = U - eta grad, formed here
            stage(s_p, U + (size_t)c0 * r, cn * r);
            stage(s_u, Gr + (size_t)c0 * r, cn * r);
        } else {
            stage(s_p, Up + (size_t)c0 * r, cn * r);
        }
        cp_async_commit();
        cp_async_wait();
        __syncthreads();
        if (from_grad) {
            for (int e = threadIdx.x; e < cn * r; e += blockDim.x) s_p[e] = csub(s_p[e], cscale(s_u[e], eta));
            __syncthreads();
        }
        for (int ii = threadIdx.x; ii < cn; ii += blockDim.x) {
            float2 u1[RMAXC];
            tri_solve_row(s_p + ii * r, u1, sL, sinv, r);
#pragma unroll
            for (int l = 0; l < RMAXC; ++l)
                if (l < r) s_u[ii * r + l] = u1[l];
        }
        __syncthreads();
        tot = cadd(tot, gram_partial(s_u, cn, r, s_red));
    }
    if (threadIdx.x < np) gpart[(size_t)blockIdx.x * np + threadIdx.x] = tot;
    if (!last_block_arrive(counter)) return;
    block_reduce_rows(gpart, gridDim.x, np, sP);
    expand_pairs(sP, r, sG);
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    double dmax = 0.0;
    for (int e = lane; e < r * r; e += 32) {
        const int a = e / r, b = e - a * r;
        const double dr = sG[2 * e] - (a == b ? 1.0 : 0.0), di = sG[2 * e + 1];
        dmax = fmax(dmax, fmax(fabs(dr), fabs(di)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (dmax <= 1e-6) {
        for (int e = lane; e < r * r; e += 32) {  // M2 = I - up(D)
            const int a = e / r, b = e - a * r;
            float2 m = make_float2(0.f, 0.f);
            if (a == b) m.x = (float)(1.0 - 0.5 * (sG[2 * e] - 1.0));
            else if (a < b) m = make_float2((float)-sG[2 * e], (float)-sG[2 * e + 1]);
            M[e] = m;
        }
        return;
    }
    // full FP64 factorisation: U1^H U1 = L2 L2^H, M2 = (L2^H)^{-1}; lane b forms column b
    const bool ok = warp_cholesky_rl(sG, r, sD);
    if (!ok) {
        if (lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_QR);
        for (int e = lane; e < r * r; e += 32) M[e] = make_float2(e / r == e % r ? 1.f : 0.f, 0.f);
        return;
    }
    if (lane < r) {
        const int b = lane;
        for (int a = r - 1; a >= 0; --a) {
            double xr = 0.0, xi = 0.0;
            if (a == b) {
                xr = sD[b];
            } else if (a < b) {  // X[a][b] = -(sum_{m=a+1..b} R2[a][m] X[m][b]) / R2[a][a], R2[a][m] = conj(L2[m][a])
                double sr = 0.0, si = 0.0;
                for (int m = a + 1; m <= b; ++m) {
                    const double lr = sG[(m * r + a) * 2], li = -sG[(m * r + a) * 2 + 1];
                    const double yr = sX[(m * r + b) * 2], yi = sX[(m * r + b) * 2 + 1];
                    sr += lr * yr - li * yi;
                    si += lr * yi + li * yr;
                }
                xr = -sr * sD[a];
                xi = -si * sD[a];
            }
            sX[(a * r + b) * 2] = xr;
            sX[(a * r + b) * 2 + 1] = xi;
        }
    }
    __syncwarp();
    for (int e = lane; e < r * r; e += 32) M[e] = make_float2((float)sX[2 * e], (float)sX[2 * e + 1]);
}

// H: U_t = U+ R1^{-1} M2 (CholeskyQR2); U_{t-1} kept in Uprev; partials of
// U_{t-1}^H U_t (for SD) and of U_t^H Z (the next iteration's h_k).
#define HMAX 8   // (k, l) pairs per thread: q r <= 256 * 8
__global__ void __launch_bounds__(NT) k_apply(float2 *__restrict__ U, float2 *__restrict__ Uprev,
                                               const float2 *__restrict__ Up, const float2 *__restrict__ Gr,
                                               const double *__restrict__ R1, const float2 *__restrict__ M,
                                               const float2 *__restrict__ Z, float2 *__restrict__ Hpart,
                                               float2 *gpart, unsigned int *counter, double *scal, int n, int r,
                                               int q, int chunk, int mode_iter) {
    extern __shared__ __align__(16) float2 smem[];
    float2 *s_up = smem;                  // chunk * r
    float2 *s_old = s_up + chunk * r;     // chunk * r
    float2 *s_new = s_old + chunk * r;    // chunk * r
    float2 *s_z = s_new + chunk * r;      // chunk * q
    __shared__ float2 sM[RMAXC * RMAXC];
    __shared__ float2 sL[RMAXC * RMAXC];
    __shared__ float sinv[RMAXC];
    __shared__ float2 s_red[NT];
    __shared__ double sC[RMAXC * RMAXC * 2];
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const float2 *Lf = (const float2 *)R1;
    const float *invf = (const float *)(Lf + r * r);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        sM[e] = M[e];
        sL[e] = Lf[e];
    }
    for (int e = threadIdx.x; e < r; e += blockDim.x) sinv[e] = invf[e];
    // U_{t-1}^H U_t pairs: thread = (entry c = a r + b, pixel group g)
    const int rr = r * r;
    const int KG = max(1, (int)blockDim.x / rr);
    const int ce = threadIdx.x % rr, cg = threadIdx.x / rr;
    const int ca = ce / r, cb = ce - ca * r;
    float2 cacc = make_float2(0.f, 0.f);
    float2 hacc[HMAX];
#pragma unroll
    for (int u = 0; u < HMAX; ++u) hacc[u] = make_float2(0.f, 0.f);
    const float eta = mode_iter ? (float)scal[SC_ETA] : 0.f;
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        __syncthreads();
        if (mode_iter) {          // U+ = U - eta grad, formed here
            stage(s_old, U + (size_t)c0 * r, cn * r);
            stage(s_up, Gr + (size_t)c0 * r, cn * r);
        } else {
            stage(s_up, Up + (size_t)c0 * r, cn * r);
        }
        stage(s_z, Z + (size_t)c0 * q, cn * q);
        cp_async_commit();
        cp_async_wait();
        __syncthreads();
        if (mode_iter) {
            for (int e = threadIdx.x; e < cn * r; e += blockDim.x) s_up[e] = csub(s_old[e], cscale(s_up[e], eta));
            __syncthreads();
        }
        for (int ii = threadIdx.x; ii < cn; ii += blockDim.x) {
            float2 u1[RMAXC];
            tri_solve_row(s_up + ii * r, u1, sL, sinv, r);
#pragma unroll
            for (int l = 0; l < RMAXC; ++l) {
                if (l < r) {
                    float2 v = make_float2(0.f, 0.f);
#pragma unroll
                    for (int m = 0; m < RMAXC; ++m)
                        if (m < r) cfma(v, u1[m], sM[m * r + l]);
                    s_new[ii * r + l] = v;
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
            U[(size_t)c0 * r + e] = s_new[e];
            if (mode_iter) Uprev[(size_t)c0 * r + e] = s_old[e];
        }
        if (mode_iter && cg < KG)
            for (int ii = cg; ii < cn; ii += KG) cfmac(cacc, s_old[ii * r + ca], s_new[ii * r + cb]);
#pragma unroll
        for (int u = 0; u < HMAX; ++u) {
            const int e = threadIdx.x + NT * u;
            if (e < q * r) {
                const int k = e / r, l = e - k * r;
                for (int ii = 0; ii < cn; ++ii) cfmac(hacc[u], s_new[ii * r + l], s_z[ii * q + k]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < HMAX; ++u) {
        const int e = threadIdx.x + NT * u;
        if (e < q * r) Hpart[(size_t)blockIdx.x * q * r + e] = hacc[u];
    }
    if (!mode_iter) return;
    if (cg < KG) s_red[cg * rr + ce] = cacc;
    __syncthreads();
    if (threadIdx.x < rr) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < KG; ++g) s = cadd(s, s_red[g * rr + threadIdx.x]);
        gpart[(size_t)blockIdx.x * rr + threadIdx.x] = s;
    }
    if (!last_block_arrive(counter)) return;
    block_reduce_rows(gpart, gridDim.x, rr, sC);
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int e = threadIdx.x; e < rr; e += 32) s += sC[2 * e] * sC[2 * e] + sC[2 * e + 1] * sC[2 * e + 1];
        s = warp_sum_d(s);
        if (threadIdx.x == 0) {
            const double sd2 = (double)r - s;  // SD^2 = r - ||U_{t-1}^H U_t||_F^2
            scal[SC_SD] = sqrt(sd2 > 0.0 ? sd2 : 0.0);
        }
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_solve(lrccs_ctx *c) {
    prof_begin(c, KID_SOLVE);
    k_solve<<<c->q, NT, 0, c->stream>>>(c->d_P, c->d_Hpart, c->d_lineptr, c->d_framerows, c->ny, c->r, c->q,
                                         c->ncg, c->nblk, c->d_B, c->d_status);
    prof_end(c, KID_SOLVE);
    return cudaGetLastError();
}

// Pixels staged per chunk: the whole per-block range when it fits in `budget`
// bytes of shared memory, else the largest multiple of 8 that does.
static int chunk_pixels(const lrccs_ctx *c, size_t bytes_per_pixel, size_t budget) {
    const int per = (c->n + c->nblk - 1) / c->nblk;
    size_t fit = budget / bytes_per_pixel;
    if (fit >= (size_t)per) return per;
    int ch = (int)(fit / 8) * 8;
    return ch < 8 ? 8 : ch;
}

cudaError_t launch_grad(lrccs_ctx *c) {
    const int r = c->r, q = c->q;
    const int ch = chunk_pixels(c, (2 * r + q) * sizeof(float2), 160 * 1024);
    prof_begin(c, KID_GRAD);
    k_grad<<<c->nblk, NT, (size_t)ch * (2 * r + q) * sizeof(float2), c->stream>>>(
        c->d_Up, c->d_Z, c->d_B, c->d_U, c->d_G, c->d_scal, c->d_gpart, c->d_counters + CNT_GRAD, c->d_R1inv,
        c->d_status, c->n, r, q, ch, c->prm.eta_c);
    prof_end(c, KID_GRAD);
    return cudaGetLastError();
}

// from_grad = 0 (init): U+ is given in Up and k_gd_gram forms R1.
// from_grad = 1 (iteration): k_grad has already formed R1 and U+ = U - eta grad
// is rebuilt from U and grad by the two kernels below.
cudaError_t launch_qr(lrccs_ctx *c, int from_grad) {
    const int r = c->r, q = c->q;
    const size_t budget = 96 * 1024;
    if (!from_grad) {
        const int chF = chunk_pixels(c, 2 * r * sizeof(float2), budget);
        prof_begin(c, KID_GD_GRAM);
        k_gd_gram<<<c->nblk, NT, (size_t)2 * chF * r * sizeof(float2), c->stream>>>(
            c->d_U, c->d_G, c->d_Up, c->d_scal, c->d_gpart, c->d_counters + CNT_QR1, c->d_R1inv, c->d_status,
            c->n, r, chF, 0);
        prof_end(c, KID_GD_GRAM);
    }
    const int chG = chunk_pixels(c, 2 * r * sizeof(float2), budget);
    prof_begin(c, KID_RINV_GRAM);
    k_rinv_gram<<<c->nblk, NT, (size_t)2 * chG * r * sizeof(float2), c->stream>>>(
        c->d_U, c->d_G, c->d_Up, c->d_scal, c->d_R1inv, c->d_gpart, c->d_counters + CNT_QR2, c->d_M, c->d_status,
        c->n, r, chG, from_grad);
    prof_end(c, KID_RINV_GRAM);
    const int chH = chunk_pixels(c, (3 * r + q) * sizeof(float2), 2 * budget);
    prof_begin(c, KID_APPLY);
    k_apply<<<c->nblk, NT, (size_t)chH * (3 * r + q) * sizeof(float2), c->stream>>>(
        c->d_U, c->d_Uprev, c->d_Up, c->d_G, c->d_R1inv, c->d_M, c->d_Z, c->d_Hpart, c->d_gpart,
        c->d_counters + CNT_APPLY, c->d_scal, c->n, r, q, chH, from_grad);
    prof_end(c, KID_APPLY);
    return cudaGetLastError();
}

cudaError_t configure_kernels_small(int max_smem) {
    cudaError_t e = allow_smem(k_gd_gram, max_smem);
    if (e == cudaSuccess) e = allow_smem(k_grad, max_smem);
    if (e == cudaSuccess) e = allow_smem(k_rinv_gram, max_smem);
    if (e == cudaSuccess) e = allow_smem(k_apply, max_smem);
    return e;
}
