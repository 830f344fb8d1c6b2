// kernels_solve.cu -- the B-step of an altGDmin iteration (Alg. 2): for each
// frame k the r x r least squares  G_k b_k = h_k  with
//   G_k = (A_k U)^H (A_k U) = sum over the frame's sampled rows ky of the
//         coil-summed row Grams P[ky] (k_row_gram),
//   h_k = (A_k U)^H y_k = U^H Z[:, k] (the per-block partial sums left by
//         k_gdqr, added here in block order),
// solved by an FP32 Cholesky factorisation, one block per frame.
#include <math.h>

#include "common.cuh"
#include "internal.h"

#define RMAXC 16   // compile-time bound on the rank
#define NT 256     // threads per block

// h_k = U^H Z[:, k] from the P partial rows of k_gdqr (hpart[b][k r + l]):
// thread (l, slice s) adds rows b = s, s + S, ... as compensated FP32 pairs,
// then lane l of the first warp adds the slices in order.  The rows are
// loaded first (frame_h_load, before the Gram sums, so that their latency
// overlaps that work) and reduced afterwards (frame_h); every thread of the
// block calls both; lanes l < R of warp 0 return h_k[l].
#define HMAX 16   // rows per thread: P <= HMAX NT / R for every R <= 16 (P <= 256)
template <int R>
static __device__ void frame_h_load(const float2 *hpart, int P, int q, int k, float2 (&v)[HMAX]) {
    constexpr int S = NT / R;
    const int t = threadIdx.x, l = t % R, s = t / R;
#pragma unroll
    for (int i = 0; i < HMAX; ++i) {
        const int b = s + i * S;
        v[i] = (s < S && b < P) ? __ldg(hpart + ((size_t)b * q + k) * R + l) : make_float2(0.f, 0.f);
    }
}
template <int R>
static __device__ float2 frame_h(const float2 (&v)[HMAX], int P, float4 *s_h) {
    constexpr int S = NT / R;
    const int t = threadIdx.x, l = t % R, s = t / R;
    if (s < S) {
        fsum2 re = {0.f, 0.f}, im = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < HMAX; ++i) {
            if (s + i * S < P) {
                fsum_add(re, v[i].x);
                fsum_add(im, v[i].y);
            }
        }
        s_h[s * R + l] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    float2 h = make_float2(0.f, 0.f);
    if (t < R) {
        fsum2 re = {0.f, 0.f}, im = {0.f, 0.f};
        for (int ss = 0; ss < S; ++ss) {
            const float4 w = s_h[ss * R + t];
            re = fsum_pair(re, fsum2{w.x, w.y});
            im = fsum_pair(im, fsum2{w.z, w.w});
        }
        h = make_float2(re.hi + re.lo, im.hi + im.lo);
    }
    return h;
}

// The Cholesky solve of one frame's r x r system from its Gram pairs sP (FP64
// sums) and h_k, by the block's first warp.
template <int R>
static __device__ void solve_frame(const double *sP, float2 *sG, float *sinv, bool any, const float2 (&hv)[HMAX],
                                   int P, int k, float4 *s_h, float2 *B, unsigned int *status) {
    constexpr int rr = R * R;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int a = e / R, b = e - a * R;
        const int p = a <= b ? pair_index(a, b, R) : pair_index(b, a, R);
        sG[e] = make_float2((float)sP[2 * p], (float)(a <= b ? sP[2 * p + 1] : -sP[2 * p + 1]));
    }
    const float2 h = frame_h<R>(hv, P, s_h);   // its barrier also publishes sG
    if ((threadIdx.x >> 5) != 0) return;
    const int lane = threadIdx.x & 31;
    const bool ok = any && warp_chol32<R>(sG, R, sinv);
    float2 x = make_float2(0.f, 0.f);
    if (ok) x = warp_chol_solve32(sG, sinv, R, h);
    if (!ok && lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_LS);
    if (lane < R) B[(size_t)k * R + lane] = x;
}

// Line masks: G_k = sum over the frame's sampled rows of the row Grams P[ky].
template <int R>
__global__ void __launch_bounds__(NT) k_solve(const float2 *__restrict__ Prow, const float2 *__restrict__ hpart,
                                              int P, int q, const int32_t *__restrict__ lineptr,
                                              const int32_t *__restrict__ framerows, float2 *__restrict__ B,
                                              unsigned int *status) {
    constexpr int np = R * (R + 1) / 2;
    __shared__ double sP[2 * np];
    __shared__ float2 sG[R * R];
    __shared__ float sinv[R];
    __shared__ int s_rows[256];
    __shared__ float4 s_h[NT];
    const int k = blockIdx.x;
    float2 hv[HMAX];
    frame_h_load<R>(hpart, P, q, k, hv);
    const int lp = lineptr[k], L = lineptr[k + 1] - lp;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s_rows[i] = framerows[lp + i];
    __syncthreads();
    // G_k pairs: sum over the frame's rows of the coil-summed row Grams
    block_sum(np, L, sP, [=](int p, int i) { return __ldg(Prow + (size_t)s_rows[i] * np + p); });
    solve_frame<R>(sP, sG, sinv, L > 0, hv, P, k, s_h, B, status);
}

// General masks: G_k = sum over the frame's samples s of the point Grams
// P_{u(s)} (u(s) = fu[s], the union index of sample s).  A frame holds
// thousands of samples, so the sum is split: block (k, c) sums chunk c of
// GEN_NCH of the frame's samples (FP64 pairs), and k_solve_gen adds the
// chunks in order and solves.
#define GEN_NCH 8
template <int R>
__global__ void __launch_bounds__(NT) k_frame_gram_gen(const float2 *__restrict__ Pu, const int32_t *__restrict__ fpk,
                                                       const int32_t *__restrict__ fu, double *__restrict__ part) {
    constexpr int np = R * (R + 1) / 2;
    const int k = blockIdx.x, c = blockIdx.y;
    const int f0 = fpk[k], m = fpk[k + 1] - f0;
    const int a0 = (int)((long long)m * c / GEN_NCH), a1 = (int)((long long)m * (c + 1) / GEN_NCH);
    const int32_t *fk = fu + f0 + a0;
    block_sum(np, a1 - a0, part + ((size_t)k * GEN_NCH + c) * 2 * np,
              [=](int p, int i) { return __ldg(Pu + (size_t)__ldg(fk + i) * np + p); });
}

template <int R>
__global__ void __launch_bounds__(NT) k_solve_gen(const double *__restrict__ part, const float2 *__restrict__ hpart,
                                                  int P, int q, const int32_t *__restrict__ fpk, float2 *__restrict__ B,
                                                  unsigned int *status) {
    constexpr int np = R * (R + 1) / 2;
    __shared__ double sP[2 * np];
    __shared__ float2 sG[R * R];
    __shared__ float sinv[R];
    __shared__ float4 s_h[NT];
    const int k = blockIdx.x;
    float2 hv[HMAX];
    frame_h_load<R>(hpart, P, q, k, hv);
    const int m = fpk[k + 1] - fpk[k];
    for (int e = threadIdx.x; e < 2 * np; e += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < GEN_NCH; ++c) acc += part[((size_t)k * GEN_NCH + c) * 2 * np + e];
        sP[e] = acc;
    }
    __syncthreads();
    solve_frame<R>(sP, sG, sinv, m > 0, hv, P, k, s_h, B, status);
}

typedef void (*solve_kernel_t)(const float2 *, const float2 *, int, int, const int32_t *, const int32_t *, float2 *,
                               unsigned int *);
static const solve_kernel_t kSolve[RMAXC] = {k_solve<1>,  k_solve<2>,  k_solve<3>,  k_solve<4>,
                                             k_solve<5>,  k_solve<6>,  k_solve<7>,  k_solve<8>,
                                             k_solve<9>,  k_solve<10>, k_solve<11>, k_solve<12>,
                                             k_solve<13>, k_solve<14>, k_solve<15>, k_solve<16>};

typedef void (*fgram_t)(const float2 *, const int32_t *, const int32_t *, double *);
typedef void (*solve_gen_t)(const double *, const float2 *, int, int, const int32_t *, float2 *, unsigned int *);
#define RANK_TABLE(K) {K<1>, K<2>, K<3>, K<4>, K<5>, K<6>, K<7>, K<8>, K<9>, K<10>, K<11>, K<12>, K<13>, K<14>, K<15>, K<16>}
static const fgram_t kFrameGramGen[RMAXC] = RANK_TABLE(k_frame_gram_gen);
static const solve_gen_t kSolveGen[RMAXC] = RANK_TABLE(k_solve_gen);

size_t frame_gram_part_count(int q, int rmax) { return (size_t)q * GEN_NCH * rmax * (rmax + 1); }

cudaError_t launch_solve(lrccs_ctx *c) {
    if (c->r < 1 || c->r > RMAXC) return cudaErrorInvalidValue;
    if (c->gd_grid > HMAX * (NT / c->r)) return cudaErrorInvalidConfiguration;   // frame_h_load's reach
    if (c->general) {
        prof_begin(c, KID_SOLVE_GEN);
        kFrameGramGen[c->r - 1]<<<dim3(c->q, GEN_NCH), NT, 0, c->stream>>>(c->d_Pu, c->d_fpk, c->d_fu, c->d_fpart);
        prof_end(c, KID_SOLVE_GEN);
        prof_begin(c, KID_SOLVE_GEN);
        kSolveGen[c->r - 1]<<<c->q, NT, 0, c->stream>>>(c->d_fpart, c->d_hpart, c->gd_grid, c->q, c->d_fpk,
                                                        c->d_B, c->d_status);
        prof_end(c, KID_SOLVE_GEN);
        return cudaGetLastError();
    }
    prof_begin(c, KID_SOLVE);
    kSolve[c->r - 1]<<<c->q, NT, 0, c->stream>>>(c->d_P, c->d_hpart, c->gd_grid, c->q, c->d_lineptr,
                                                 c->d_framerows, c->d_B, c->d_status);
    prof_end(c, KID_SOLVE);
    return cudaGetLastError();
}
