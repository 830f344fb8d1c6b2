// kernels_solve.cu -- the B-step of an altGDmin iteration (Alg. 2): for each
// frame k the r x r least squares  G_k b_k = h_k  with
//   G_k = (A_k U)^H (A_k U) = sum over the frame's sampled rows ky of the
//         coil-summed row Grams P[ky] (k_row_gram),
//   h_k = (A_k U)^H y_k = U^H Z[:, k] (the per-block partial sums left by
//         k_gdqr, added here in block order),
// solved in FP32 by Gauss-Jordan elimination (one warp), one block per frame.
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

// Warp 0: b_k = G_k^{-1} h_k by Gauss-Jordan elimination of [G_k | h_k]
// without pivoting (G_k is Hermitian positive definite, so the pivots are the
// positive diagonal of its LDL^H factorisation), lane i holding row i in
// registers: one broadcast of the pivot row per step, no separate triangular
// solves.  A pivot that is not positive marks the frame rank deficient
// (ST_NOT_SPD_LS, b_k = 0).  Not inlined, so that its registers are allocated
// on their own inside the large fused kernel.
template <int R>
static __device__ __noinline__ void gj_solve_warp(const float2 *sG, bool any, float2 h, int k, float2 *B,
                                                  unsigned int *status) {
    const int lane = threadIdx.x & 31;
    float2 m[R + 1];
#pragma unroll
    for (int j = 0; j < R; ++j) m[j] = lane < R ? sG[lane * R + j] : make_float2(0.f, 0.f);
    m[R] = lane < R ? h : make_float2(0.f, 0.f);
    bool ok = any;
#pragma unroll
    for (int c = 0; c < R; ++c) {
        const float piv = __shfl_sync(0xffffffffu, m[c].x, c);
        ok = ok && piv > 0.f;
        const float inv = ok ? 1.f / piv : 0.f;
        float2 pr[R + 1];
#pragma unroll
        for (int j = c + 1; j <= R; ++j)
            pr[j] = make_float2(__shfl_sync(0xffffffffu, m[j].x, c), __shfl_sync(0xffffffffu, m[j].y, c));
        if (lane == c) {
#pragma unroll
            for (int j = c + 1; j <= R; ++j) m[j] = cscale(m[j], inv);
        } else {
            const float2 f = cscale(m[c], inv);   // G[i][c] / pivot
#pragma unroll
            for (int j = c + 1; j <= R; ++j) m[j] = csub(m[j], cmul(f, pr[j]));
        }
    }
    if (!ok && lane == 0) atomicOr(status, (unsigned)ST_NOT_SPD_LS);
    if (lane < R) B[(size_t)k * R + lane] = ok ? m[R] : make_float2(0.f, 0.f);
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
    gj_solve_warp<R>(sG, any, h, k, B, status);
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

// ---------------------------------------------------------------- fused B-step over resident rows
//
// k_bstep does the line-mask B-step and the row weighting of the gradient in
// one cooperative launch, one block per sampled row (every row resident in
// shared memory for the whole launch, so T is read once and written once):
//   phase A  row ky: bulk copies of T_j[ky] (one mbarrier per coil), the
//            coil-summed row Gram P[ky] = sum_j sum_x T_j[ky][x]^H T_j[ky][x];
//   barrier
//   phase B  frame k = block, block + G, ...: G_k = sum of its rows' P, h_k
//            from k_gdqr's partial rows, FP32 Cholesky -> b_k (as k_solve);
//   barrier
//   phase C  row ky: W_ky = sum over the frames sampling ky of b_k b_k^H, then
//            T_j[ky][x][:] <- T_j[ky][x][:] W_ky from the resident row (as k_row_w);
//            every block: Z B^H for its share of the pixels (as k_zb).
// It replaces k_row_gram, k_solve, k_row_w and k_zb when every sampled row
// fits one block's shared memory and all rows' blocks are co-resident.
#define BS_NT 512     // threads per block
#define BS_MAXC 32    // coils (one mbarrier each)

// Phase A thread layout for rank R: the R x R Gram is cut into NB x NB blocks
// of edge TB; the NU blocks on or above the diagonal each get a share of the
// 16 warps in proportion to their work (bs_wstart), whose lanes stride over
// the row's C nx vectors and accumulate their block in registers (NV floats,
// padded for the warp reduction).
template <int R>
struct BsPlan {
    static constexpr int NB = (R + 4) / 5;
    static constexpr int TB = (R + NB - 1) / NB;
    static constexpr int NU = NB * (NB + 1) / 2;
    static constexpr int NV = 2 * TB * TB <= 32 ? 32 : 64;
};
__host__ __device__ constexpr int bs_bi(int g, int nb) {
    int bi = 0;
    while (g >= nb - bi) { g -= nb - bi; ++bi; }
    return bi;
}
__host__ __device__ constexpr int bs_bj(int g, int nb) {
    int bi = 0;
    while (g >= nb - bi) { g -= nb - bi; ++bi; }
    return bi + g;
}
// complex MACs per vector of Gram block g: the upper triangle of a diagonal
// block, all of an off-diagonal one, clipped at R
__host__ __device__ constexpr int bs_work(int g, int R) {
    const int nb = (R + 4) / 5, tb = (R + nb - 1) / nb, bi = bs_bi(g, nb), bj = bs_bj(g, nb);
    int w = 0;
    for (int i = 0; i < tb; ++i)
        for (int j = 0; j < tb; ++j)
            if (bi * tb + i < R && bj * tb + j < R && (bi != bj || j >= i)) ++w;
    return w;
}
// First warp of group g (g = NU gives 16): one warp each, then every further
// warp to the group with the most work per warp (lowest g on ties).
__host__ __device__ constexpr int bs_wstart(int g, int R) {
    const int nb = (R + 4) / 5, nu = nb * (nb + 1) / 2;
    int al[10] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    for (int used = nu; used < BS_NT / 32; ++used) {
        int best = 0;
        for (int u = 1; u < nu; ++u)
            if (bs_work(u, R) * al[best] > bs_work(best, R) * al[u]) best = u;
        ++al[best];
    }
    int st = 0;
    for (int u = 0; u < g && u < nu; ++u) st += al[u];
    return st;
}

// bs_wstart(g, R) for a runtime g, from constants folded at compile time
template <int R, int U = 0>
LRCCS_DEV int bs_ws(int g) {
    if constexpr (U >= BsPlan<R>::NU) {
        return BS_NT / 32;
    } else {
        constexpr int v = bs_wstart(U, R);
        return g == U ? v : bs_ws<R, U + 1>(g);
    }
}
// the Gram block whose warps include `warp`
template <int R, int U = 0>
LRCCS_DEV int bs_group_of(int warp) {
    if constexpr (U + 1 >= BsPlan<R>::NU) {
        return U;
    } else {
        constexpr int next = bs_wstart(U + 1, R);
        return warp < next ? U : bs_group_of<R, U + 1>(warp);
    }
}

// Elements [E0, E0 + N) of one R-vector in shared memory into registers
// (zero past R); 16-byte loads when R is even (the vector starts 16-byte aligned).
template <int R, int E0, int N>
LRCCS_DEV void bs_load(const float2 *vec, float2 (&o)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) o[i] = make_float2(0.f, 0.f);
    if constexpr (R % 2 == 0) {
#pragma unroll
        for (int p = E0 & ~1; p < E0 + N && p < R; p += 2) {
            const float4 w = *reinterpret_cast<const float4 *>(vec + p);
            if (p >= E0) o[p - E0] = make_float2(w.x, w.y);
            if (p + 1 >= E0 && p + 1 < E0 + N) o[p + 1 - E0] = make_float2(w.z, w.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (E0 + i < R) o[i] = vec[E0 + i];
    }
}

// Reduce NV floats over the 32 lanes of a warp by recursive halving: after
// the five exchange steps lane L holds the sums of entries [L NV/32, (L+1) NV/32).
template <int NV>
LRCCS_DEV void bs_warp_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
    for (int m = 16, h = NV / 2; m >= 1; m >>= 1, h >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
}

// One Gram block (BI, BJ): lane (slice s of S) accumulates
// sum_v conj(T_v[BI TB + i]) T_v[BJ TB + jj] over vectors v = s, s + S, ...
// (v = j nx + x), waiting for coil j's copy before its first vector.
template <int R, int BI, int BJ>
LRCCS_DEV void bs_gram_block(const float2 *row, int nc, int nx, int s, int S, uint64_t *mbar, unsigned limit,
                             bool &late, float (&acc)[BsPlan<R>::NV]) {
    constexpr int TB = BsPlan<R>::TB;
    const int V = nc * nx;
    int j = s / nx, x = s - j * nx, jw = -1;
    for (int v = s; v < V; v += S) {
        if (j != jw) {
            if (!mbar_wait(mbar + j, 0, limit)) late = true;
            jw = j;
        }
        const float2 *vec = row + (size_t)v * R;
        float2 a[TB], b[TB];
        bs_load<R, BI * TB, TB>(vec, a);
        if constexpr (BI == BJ) {
#pragma unroll
            for (int i = 0; i < TB; ++i) b[i] = a[i];
        } else {
            bs_load<R, BJ * TB, TB>(vec, b);
        }
#pragma unroll
        for (int i = 0; i < TB; ++i)
#pragma unroll
            for (int jj = 0; jj < TB; ++jj) {
                if (BI == BJ && jj < i) continue;
                if (BI * TB + i >= R || BJ * TB + jj >= R) continue;
                float2 c = make_float2(acc[2 * (i * TB + jj)], acc[2 * (i * TB + jj) + 1]);
                cfmac(c, a[i], b[jj]);
                acc[2 * (i * TB + jj)] = c.x;
                acc[2 * (i * TB + jj) + 1] = c.y;
            }
        x += S;
        while (x >= nx) {
            x -= nx;
            ++j;
        }
    }
}

template <int R, int G>
LRCCS_DEV void bs_gram_dispatch(int g, const float2 *row, int nc, int nx, int s, int S, uint64_t *mbar,
                                unsigned limit, bool &late, float (&acc)[BsPlan<R>::NV]) {
    if constexpr (G < BsPlan<R>::NU) {
        if (g == G)
            bs_gram_block<R, bs_bi(G, BsPlan<R>::NB), bs_bj(G, BsPlan<R>::NB)>(row, nc, nx, s, S, mbar, limit, late,
                                                                               acc);
        else
            bs_gram_dispatch<R, G + 1>(g, row, nc, nx, s, S, mbar, limit, late, acc);
    }
}

// Row stride (complex values) of Z rows staged for Z B^H: the smallest
// value >= q that is 2 mod 16.
__host__ __device__ inline int bs_zstride(int q) { return q + ((18 - q % 16) % 16); }

struct BstepArgs {
    float2 *T;                    // [j][ky][x][l]: the sampled rows in, T_j[ky] W_ky out
    float2 *Prow;                 // [ky][pair] coil-summed row Grams (written in phase A)
    const float2 *hpart;          // P x q r partial rows of h = U^H Z (k_gdqr)
    const int32_t *usedrows;      // the sampled rows (block b: row usedrows[b])
    const int32_t *lineptr, *framerows;   // rows of frame k: framerows[lineptr[k] ..]
    const int32_t *rfptr, *rflist;        // frames of row ky: rflist[rfptr[ky] ..]
    float2 *B;                    // q x r (written in phase B)
    const float2 *Z;              // n x q  A_k^H y_k, row-major (i q + k)
    float2 *ZB;                   // n x r  Z B^H (written in phase C)
    unsigned int *bar;            // [0] barrier arrivals, [1] exit count
    unsigned int *status;
    int ny, nx, nc, q, P, n;      // P: partial rows of h
    unsigned int spin_limit;      // polls before a grid barrier gives up
    long long *ts;                // NULL, or BS_NTS global-timer stamps (ns) per block b < ts_blocks
    int ts_blocks;
};

// Phase timing (measurement support): thread 0 of block b stamps the global
// timer at entry, after phase A, after the first barrier, after its first
// frame's Gram sum, after phase B, after the second barrier, after W, after
// the row weighting, after the first Z chunk is staged, after Z B^H and at
// exit.
#define BS_NTS 11
#define BS_TS(i)                                                                             \
    do {                                                                                     \
        if (a.ts && threadIdx.x == 0 && (int)blockIdx.x < a.ts_blocks) {                     \
            unsigned long long g_;                                                           \
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g_));                           \
            a.ts[(size_t)blockIdx.x * BS_NTS + (i)] = (long long)g_;                         \
        }                                                                                    \
    } while (0)

template <int R>
__global__ void __launch_bounds__(BS_NT, 1) k_bstep(const __grid_constant__ BstepArgs a) {
    using PL = BsPlan<R>;
    constexpr int np = R * (R + 1) / 2, NV = PL::NV, TB = PL::TB;
    extern __shared__ __align__(128) float2 bs_smem[];
    // 128-byte aligned start (bulk-copy destination); the launch adds 128 bytes of slack
    float2 *row = (float2 *)(((uintptr_t)bs_smem + 127) & ~(uintptr_t)127);   // nc nx R: T_j[ky] of every coil
    float2 *sB = row + (size_t)a.nc * a.nx * R;             // q R
    __shared__ __align__(8) uint64_t s_mbar[BS_MAXC];
    __shared__ float s_part[(BS_NT / 32) * 64];
    __shared__ double sP[2 * np];
    __shared__ float2 sG[R * R];
    __shared__ float2 sW[R * R];
    __shared__ float sinv[R];
    __shared__ int s_rows[256];
    __shared__ int s_f[128];
    __shared__ float4 s_h[NT];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int G = gridDim.x, ky = a.usedrows[blockIdx.x];
    const int nx = a.nx, nc = a.nc, q = a.q;
    const size_t plane = (size_t)a.ny * nx * R;
    const unsigned rowbytes = (unsigned)(nx * R * sizeof(float2));

    BS_TS(0);
    // ---- phase A: the row in by bulk copies, its coil-summed Gram
    if (t == 0) {
        for (int j = 0; j < nc; ++j) mbar_init(s_mbar + j, 1);
    }
    __syncthreads();
    if (t == 0) {
        for (int j = 0; j < nc; ++j) {
            const unsigned bar = smem_u32(s_mbar + j);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(rowbytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(row + (size_t)j * nx * R)),
                "l"(a.T + (size_t)j * plane + (size_t)ky * nx * R), "r"(rowbytes), "r"(bar)
                : "memory");
        }
    }
    bool late = false;
    {
        float acc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0.f;
        const int g = bs_group_of<R>(warp);
        const int w0 = bs_ws<R>(g), nw = bs_ws<R>(g + 1) - w0;
        bs_gram_dispatch<R, 0>(g, row, nc, nx, (warp - w0) * 32 + lane, nw * 32, s_mbar, 1u << 22, late, acc);
        bs_warp_reduce_scatter<NV>(acc, lane);
#pragma unroll
        for (int u = 0; u < NV / 32; ++u) s_part[warp * 64 + lane * (NV / 32) + u] = acc[u];
    }
    if (late) atomicOr(a.status, (unsigned)ST_TIMEOUT);
    __syncthreads();
    // pair (x, y), x <= y: block (x / TB, y / TB), entry (x % TB, y % TB), summed over its warps in order
    for (int e = t; e < R * R; e += BS_NT) {
        const int x = e / R, y = e - x * R;
        if (x > y) continue;
        const int bi = x / TB, bj = y / TB;
        const int gi = bi * PL::NB - (bi * (bi - 1)) / 2 + (bj - bi);
        const int ent = (x - bi * TB) * TB + (y - bj * TB);
        float re = 0.f, im = 0.f;
        for (int w = bs_ws<R>(gi); w < bs_ws<R>(gi + 1); ++w) {
            re += s_part[w * 64 + 2 * ent];
            im += s_part[w * 64 + 2 * ent + 1];
        }
        a.Prow[(size_t)ky * np + pair_index(x, y, R)] = make_float2(re, im);
    }

    BS_TS(1);
    // ---- phase B: the per-frame solves (h rows and row lists fetched before the barrier)
    float2 hv[HMAX];
    int L = 0;
    if ((int)blockIdx.x < q) {
        const int k = blockIdx.x;
        frame_h_load<R>(a.hpart, a.P, q, k, hv);
        const int lp = a.lineptr[k];
        L = a.lineptr[k + 1] - lp;
        for (int i = t; i < L; i += BS_NT) s_rows[i] = a.framerows[lp + i];
    }
    grid_sync(a.bar, 1, a.status, a.spin_limit, 0, ST_TIMEOUT);
    BS_TS(2);
    for (int k = blockIdx.x; k < q; k += G) {
        if (k != (int)blockIdx.x) {
            frame_h_load<R>(a.hpart, a.P, q, k, hv);
            const int lp = a.lineptr[k];
            L = a.lineptr[k + 1] - lp;
            for (int i = t; i < L; i += BS_NT) s_rows[i] = a.framerows[lp + i];
            __syncthreads();
        }
        const float2 *Pr = a.Prow;
        block_sum(np, L, sP, [=](int p, int i) { return __ldcg(Pr + (size_t)s_rows[i] * np + p); });
        if (k == (int)blockIdx.x) BS_TS(3);
        solve_frame<R>(sP, sG, sinv, L > 0, hv, a.P, k, s_h, a.B, a.status);
        __syncthreads();
    }

    if ((int)blockIdx.x >= q) BS_TS(3);
    BS_TS(4);
    // ---- phase C: W_ky from the new B, applied to the resident row
    const int f0 = a.rfptr[ky], nf = a.rfptr[ky + 1] - f0;
    for (int f = t; f < nf; f += BS_NT) s_f[f] = a.rflist[f0 + f];
    grid_sync(a.bar, 2, a.status, a.spin_limit, 0, ST_TIMEOUT);
    BS_TS(5);
    for (int e = t; e < q * R; e += BS_NT) sB[e] = __ldcg(a.B + e);
    __syncthreads();
    for (int e = t; e < R * R; e += BS_NT) {
        const int x = e / R, y = e - x * R;
        float2 acc = make_float2(0.f, 0.f);
        for (int f = 0; f < nf; ++f) cfma(acc, sB[s_f[f] * R + x], cconj(sB[s_f[f] * R + y]));
        sW[e] = acc;
    }
    __syncthreads();
    BS_TS(6);
    {
        constexpr int OC = (R % 2 == 0) ? 2 : 1;   // output columns per thread
        constexpr int NTPV = R / OC;               // threads per vector
        constexpr int NG = BS_NT / NTPV;           // vector groups
        const int wo = t % NTPV, vg = t / NTPV;
        if (vg < NG) {
            float2 wc[OC][R];
#pragma unroll
            for (int o = 0; o < OC; ++o)
#pragma unroll
                for (int x = 0; x < R; ++x) wc[o][x] = sW[x * R + wo * OC + o];
            const int V = nc * nx;
            // two vectors per step (v and v + NG): twice the independent FMA chains
            auto store = [&](int j, int x, const float2 (&out)[OC]) {
                float2 *dst = a.T + (size_t)j * plane + ((size_t)ky * nx + x) * R + wo * OC;
                if constexpr (OC == 2) *reinterpret_cast<float4 *>(dst) = make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
                else *dst = out[0];
            };
            int j = vg / nx, x = vg - j * nx;
            for (int v = vg; v < V; v += 2 * NG) {
                int j2 = j, x2 = x + NG;
                while (x2 >= nx) {
                    x2 -= nx;
                    ++j2;
                }
                const bool has2 = v + NG < V;
                float2 in1[R], in2[R];
                bs_load<R, 0, R>(row + (size_t)v * R, in1);
                bs_load<R, 0, R>(row + (size_t)(has2 ? v + NG : v) * R, in2);
                float2 out1[OC], out2[OC];
#pragma unroll
                for (int o = 0; o < OC; ++o) {
                    out1[o] = make_float2(0.f, 0.f);
                    out2[o] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int y = 0; y < R; ++y) {
                        cfma(out1[o], in1[y], wc[o][y]);
                        cfma(out2[o], in2[y], wc[o][y]);
                    }
                }
                store(j, x, out1);
                if (has2) store(j2, x2, out2);
                j = j2;
                x = x2 + NG;
                while (x >= nx) {
                    x -= nx;
                    ++j;
                }
            }
        }
    }
    BS_TS(7);
    // ---- Z B^H for this block's share of the pixels (the data term of the
    // next gradient).  The pixels' Z rows are staged in chunks into the row
    // buffer (free after the weighting) with a row stride of 2 mod 16 complex
    // values, so that the 16 lanes of a half-warp read distinct bank pairs of
    // Z.  Each thread keeps all R outputs of two pixels in registers, so every
    // row of B read (a broadcast) serves two pixels.
    {
        const int per = (a.n + G - 1) / G, i0 = blockIdx.x * per, i1 = min(a.n, i0 + per);
        const int qs = bs_zstride(q);                // staged row stride
        const int cap = (nc * nx * R) / qs;          // pixels per chunk
        float2 *zs = row;
        for (int c0 = i0; c0 < i1; c0 += cap) {
            const int c1 = min(i1, c0 + cap), np_ = c1 - c0, cnt = np_ * q;
            const float2 *src = a.Z + (size_t)c0 * q;
            __syncthreads();   // the previous users of the buffer are done
            // element e = pi q + k of the chunk -> zs[pi qs + k], indices stepped
            // without division; 16-byte copies of (k, k + 1) pairs when q is
            // even (qs is even, so both sides are 16-byte aligned)
            const int w = (q & 1) ? 1 : 2, qw = q / w, cw = cnt / w;
            const int dpi = BS_NT / qw, dk = BS_NT - dpi * qw;
            int pi = t / qw, k = t - pi * qw;
            for (int e = t; e < cw; e += BS_NT) {
                if (w == 2) cp_async16(zs + pi * qs + 2 * k, src + 2 * e);
                else cp_async8(zs + pi * qs + k, src + e);
                pi += dpi;
                k += dk;
                if (k >= qw) {
                    k -= qw;
                    ++pi;
                }
            }
            cp_async_commit();
            cp_async_wait();
            __syncthreads();
            if (c0 == i0) BS_TS(8);
            // thread (pixel pair pp, quarter m): pixels 2pp and 2pp + 1 of the
            // chunk over the frames k = m, m + 4, ...; the four quarters are
            // added by shuffles and lane m writes the outputs l = m, m + 4, ...
            const int m4 = t & 3, npair = (np_ + 1) >> 1;
            for (int pp = t >> 2; pp < ((npair + 7) & ~7); pp += BS_NT / 4) {   // whole warps take part
                const int p0 = 2 * pp, p1 = p0 + 1;
                const bool live0 = p0 < np_, live1 = p1 < np_;
                float2 acc0[R], acc1[R];
#pragma unroll
                for (int l = 0; l < R; ++l) acc0[l] = acc1[l] = make_float2(0.f, 0.f);
                if (live0) {
                    const float2 *z0r = zs + p0 * qs, *z1r = zs + (live1 ? p1 : p0) * qs;
                    for (int k = m4; k < q; k += 4) {
                        const float2 z0 = z0r[k], z1 = live1 ? z1r[k] : make_float2(0.f, 0.f);
                        float2 br[R];
                        bs_load<R, 0, R>(sB + k * R, br);   // 16-byte loads for even R
#pragma unroll
                        for (int l = 0; l < R; ++l) {
                            const float2 bc = cconj(br[l]);
                            cfma(acc0[l], z0, bc);
                            cfma(acc1[l], z1, bc);
                        }
                    }
                }
#pragma unroll
                for (int l = 0; l < R; ++l) {
                    acc0[l] = cadd(acc0[l], shfl_xor2(acc0[l], 1));
                    acc1[l] = cadd(acc1[l], shfl_xor2(acc1[l], 1));
                    acc0[l] = cadd(acc0[l], shfl_xor2(acc0[l], 2));
                    acc1[l] = cadd(acc1[l], shfl_xor2(acc1[l], 2));
                }
#pragma unroll
                for (int l = 0; l < R; ++l) {
                    if ((l & 3) != m4) continue;
                    if (live0) a.ZB[(size_t)(c0 + p0) * R + l] = acc0[l];
                    if (live1) a.ZB[(size_t)(c0 + p1) * R + l] = acc1[l];
                }
            }
        }
    }

    // the last block out returns the barrier counters to zero (every block is past its last barrier)
    __shared__ bool s_last;
    __syncthreads();
    BS_TS(9);
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(a.bar + 1, 1u) == (unsigned)G - 1;
        if (s_last) {
            a.bar[0] = 0u;
            a.bar[1] = 0u;
        }
    }
    BS_TS(10);
}

typedef void (*bstep_kernel_t)(const BstepArgs);
static const bstep_kernel_t kBstep[RMAXC] = RANK_TABLE(k_bstep);

static size_t bstep_smem(int nc, int nx, int q, int r) {
    return ((size_t)nc * nx * r + (size_t)q * r) * sizeof(float2) + 128;
}

cudaError_t configure_kernels_solve(int max_smem) {
    for (int i = 0; i < RMAXC; ++i) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kBstep[i]);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kBstep[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Blocks of k_bstep<r> that can be resident at once for this shape (0: one
// sampled row does not fit a block's shared memory, or too many coils).
int bstep_capacity(int nc, int nx, int q, int r, int smem_optin, int nsm) {
    if (r < 1 || r > RMAXC || nc < 1 || nc > BS_MAXC || q < 1 || q > 128 || ((size_t)nx * r) % 2 != 0) return 0;
    if ((size_t)nc * nx * r < (size_t)bs_zstride(q)) return 0;   // Z B^H stages whole Z rows in the row buffer
    const size_t smem = bstep_smem(nc, nx, q, r);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kBstep[r - 1]) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (smem + fa.sharedSizeBytes > (size_t)smem_optin) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kBstep[r - 1], BS_NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb * nsm;
}

// The fused form applies to line masks when every sampled row gets its own
// resident block (and the plan does not ask for the separate kernels).
bool bstep_fused_ok(const lrccs_ctx *c) {
    if (c->plan.bstep_form != 0 || c->general || c->r < 1 || c->r > RMAXC) return false;
    if (c->gd_grid > HMAX * (NT / c->r)) return false;   // frame_h_load's reach
    return c->n_used >= 1 && c->n_used <= c->bs_cap[c->r];
}

// B (row Grams, per-frame solves), the row weighting T_j[ky] W_ky and Z B^H
// in one cooperative launch (replaces k_row_gram, k_solve, k_row_w and k_zb).
cudaError_t launch_bstep_fused(lrccs_ctx *c) {
    const int r = c->r;
    if (!bstep_fused_ok(c)) return cudaErrorInvalidConfiguration;
    BstepArgs a;
    a.T = c->d_T;
    a.Prow = c->d_P;
    a.hpart = c->d_hpart;
    a.usedrows = c->d_usedrows;
    a.lineptr = c->d_lineptr;
    a.framerows = c->d_framerows;
    a.rfptr = c->d_rfptr;
    a.rflist = c->d_rflist;
    a.B = c->d_B;
    a.Z = c->d_Z;
    a.ZB = c->d_ZB;
    a.n = c->n;
    a.bar = c->d_counters + CNT_BS_BAR;
    a.status = c->d_status;
    a.ny = c->ny;
    a.nx = c->nx;
    a.nc = c->nc;
    a.q = c->q;
    a.P = c->gd_grid;
    a.spin_limit = 1u << 24;
    // phase stamps after k_gdqr's in the phase-timing buffer (lrccs_gdqr_phases on)
    a.ts = c->d_gdts ? c->d_gdts + (size_t)c->gd_grid * 11 : nullptr;
    a.ts_blocks = c->gd_grid;
    void *args[] = {&a};
    prof_begin(c, KID_BSTEP);
    const cudaError_t e = cudaLaunchCooperativeKernel((const void *)kBstep[r - 1], dim3(c->n_used), dim3(BS_NT), args,
                                                      bstep_smem(c->nc, c->nx, c->q, r), c->stream);
    prof_end(c, KID_BSTEP);
    return e;
}
