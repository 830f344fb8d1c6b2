// kernels_iter.cu -- one altGDmin iteration (Alg. 2, GDmin loop) on sm_103a.
//
// The iteration uses three exact rearrangements of Alg. 2 (linearity only):
//   A_k U = H_k [F(d_j o U)]_j         -> C r forward 2D transforms per iteration,
//                                          shared by every frame;
//   (A_k U)^H y_k = U^H Z[:, k]         -> the right-hand side never re-reads y;
//   sum_k A_k^H (A_k U b_k - y_k) b_k^H
//     = sum_j conj(d_j) o F^H [FU_j[i,:] W_i] - Z B^H,   W_i = sum_{k: i in Omega_k} b_k b_k^H
//                                        -> C r inverse transforms per iteration.
// With line masks W_i and the Gram contributions are constant along a sampled
// row ky, so they are formed once per row.
//
// Kernels (one launch each per iteration):
//   A k_fwd_cols  : F_y of d_j o U over column tiles               -> T[j][ky][x][l]
//   B k_fwd_rows  : F_x of every sampled row, row Gram partials    -> FU (in place), P
//   C k_solve     : G_k = sum of its rows' P, h_k, FP64 Cholesky    -> B
//   D k_adj_rows  : K = FU W_ky, F_x^H                              -> T (in place)
//   E k_adj_cols  : F_y^H, conj(d_j) coil sum, - Z B^H              -> grad; eta at t = 1
//   F k_gd_gram   : U+ = U - eta grad, Gram of U+, Cholesky         -> R1^{-1}
//   G k_rinv_gram : Gram of U+ R1^{-1}, Cholesky                   -> M = R1^{-1} R2^{-1}
//   H k_apply     : U_t = U+ M (CholeskyQR2), SD, next h partials
#include <math.h>

#include "common.cuh"
#include "internal.h"

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

#define RMAXC 16   // compile-time bound on the rank

int npairs_of(int r) { return r * (r + 1) / 2; }

static inline int pitch_odd(int c) { return c | 1; }

// ---------------------------------------------------------------- A: forward, along y

template <int P>
__global__ void __launch_bounds__(256) k_fwd_cols(const float2 *__restrict__ U, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, float2 *__restrict__ T,
                                                   int nx, int r, int tx, const float2 *__restrict__ g_tw,
                                                   float scale) {
    constexpr int NY = 32 * P;
    extern __shared__ float2 smem[];
    float2 *s_tw = smem;
    float2 *tile = smem + NY;
    const int C = tx * r, TP = C | 1;
    const int x0 = blockIdx.x * tx, j = blockIdx.y;
    const size_t n = (size_t)NY * nx;
    load_twiddles(s_tw, g_tw, NY);
    const float2 *Uc = U + (size_t)x0 * r;
    const float2 *Sj = smaps + (size_t)j * n + x0;
    for (int e = threadIdx.x; e < NY * C; e += blockDim.x) {
        const int y = e / C, c = e - y * C;
        tile[y * TP + c] = cmul(Sj[(size_t)y * nx + c / r], Uc[(size_t)y * nx * r + c]);
    }
    __syncthreads();
    tile_fft<P>(tile, TP, 1, C, s_tw, false, scale);
    __syncthreads();
    float2 *Tj = T + ((size_t)j * n + x0) * r;
    for (int e = threadIdx.x; e < NY * C; e += blockDim.x) {
        const int ky = e / C, c = e - ky * C;
        if (rowused[ky]) Tj[(size_t)ky * nx * r + c] = tile[ky * TP + c];
    }
}

// ---------------------------------------------------------------- B: forward, along x + row Gram

template <int P>
__global__ void __launch_bounds__(256) k_fwd_rows(float2 *__restrict__ T, const int32_t *__restrict__ usedrows,
                                                   float2 *__restrict__ Ppart, int ny, int r, int nc, int cpg,
                                                   const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * P;
    extern __shared__ float2 smem[];
    float2 *s_tw = smem;
    float2 *tile = s_tw + NX;
    const int RP = r | 1;
    float2 *s_red = tile + NX * RP;
    const int ky = usedrows[blockIdx.x], g = blockIdx.y;
    const int j0 = g * cpg, j1 = min(nc, j0 + cpg);
    const size_t n = (size_t)ny * NX;
    const int np = r * (r + 1) / 2;
    const int KG = max(1, (int)blockDim.x / np);
    const int p = threadIdx.x % np, kg = threadIdx.x / np;
    const bool active = kg < KG;
    int a = 0, b = 0;
    pair_of(p, r, a, b);
    float2 acc = make_float2(0.f, 0.f);
    load_twiddles(s_tw, g_tw, NX);
    for (int j = j0; j < j1; ++j) {
        __syncthreads();
        float2 *row = T + ((size_t)j * n + (size_t)ky * NX) * r;
        for (int e = threadIdx.x; e < NX * r; e += blockDim.x) {
            const int x = e / r, l = e - x * r;
            tile[x * RP + l] = row[e];
        }
        __syncthreads();
        tile_fft<P>(tile, RP, 1, r, s_tw, false, scale);
        __syncthreads();
        for (int e = threadIdx.x; e < NX * r; e += blockDim.x) {
            const int x = e / r, l = e - x * r;
            row[e] = tile[x * RP + l];
        }
        if (active)
            for (int kx = kg; kx < NX; kx += KG) cfmac(acc, tile[kx * RP + a], tile[kx * RP + b]);
    }
    __syncthreads();
    if (active) s_red[kg * np + p] = acc;
    __syncthreads();
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < KG; ++q) s = cadd(s, s_red[q * np + pp]);
        Ppart[((size_t)g * ny + ky) * np + pp] = s;
    }
}

// ---------------------------------------------------------------- C: per-frame LS (FP64 Cholesky)
// G_k b_k = h_k with G_k = (A_k U)^H (A_k U) = sum over the frame's rows of P,
// h_k = U^H Z[:, k] (Alg. 2, B-update).

__global__ void k_solve(const float2 *__restrict__ Ppart, const float2 *__restrict__ Hpart,
                        const int32_t *__restrict__ lineptr, const int32_t *__restrict__ framerows, int ny, int r,
                        int q, int ncg, int nblkH, float2 *__restrict__ B, unsigned int *status) {
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sh[RMAXC * 2];
    const int k = blockIdx.x;
    const int np = r * (r + 1) / 2;
    const int lp = lineptr[k], L = lineptr[k + 1] - lp;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < L; ++i) {
            const int ky = framerows[lp + i];
            for (int g = 0; g < ncg; ++g) {
                const float2 v = Ppart[((size_t)g * ny + ky) * np + p];
                re += v.x;
                im += v.y;
            }
        }
        int a, b;
        pair_of(p, r, a, b);
        sG[(a * r + b) * 2] = re;
        sG[(a * r + b) * 2 + 1] = im;
        sG[(b * r + a) * 2] = re;
        sG[(b * r + a) * 2 + 1] = -im;
    }
    for (int l = threadIdx.x; l < r; l += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int blk = 0; blk < nblkH; ++blk) {
            const float2 v = Hpart[((size_t)blk * q + k) * r + l];
            re += v.x;
            im += v.y;
        }
        sh[2 * l] = re;
        sh[2 * l + 1] = im;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // Cholesky G = L L^H, L lower, stored in place of the lower triangle of sG
    bool ok = L > 0;
    for (int c = 0; c < r && ok; ++c) {
        double d = sG[(c * r + c) * 2];
        for (int m = 0; m < c; ++m) d -= sG[(c * r + m) * 2] * sG[(c * r + m) * 2] + sG[(c * r + m) * 2 + 1] * sG[(c * r + m) * 2 + 1];
        if (!(d > 0.0)) { ok = false; break; }
        d = sqrt(d);
        sG[(c * r + c) * 2] = d;
        sG[(c * r + c) * 2 + 1] = 0.0;
        for (int rr = c + 1; rr < r; ++rr) {
            double vr = sG[(rr * r + c) * 2], vi = sG[(rr * r + c) * 2 + 1];
            for (int m = 0; m < c; ++m) {
                // v -= L[rr][m] conj(L[c][m])
                const double ar = sG[(rr * r + m) * 2], ai = sG[(rr * r + m) * 2 + 1];
                const double br = sG[(c * r + m) * 2], bi = sG[(c * r + m) * 2 + 1];
                vr -= ar * br + ai * bi;
                vi -= ai * br - ar * bi;
            }
            sG[(rr * r + c) * 2] = vr / d;
            sG[(rr * r + c) * 2 + 1] = vi / d;
        }
    }
    double z[2 * RMAXC];
    if (ok) {
        for (int c = 0; c < r; ++c) {  // L z = h
            double vr = sh[2 * c], vi = sh[2 * c + 1];
            for (int m = 0; m < c; ++m) {
                const double ar = sG[(c * r + m) * 2], ai = sG[(c * r + m) * 2 + 1];
                vr -= ar * z[2 * m] - ai * z[2 * m + 1];
                vi -= ar * z[2 * m + 1] + ai * z[2 * m];
            }
            const double d = sG[(c * r + c) * 2];
            z[2 * c] = vr / d;
            z[2 * c + 1] = vi / d;
        }
        for (int c = r - 1; c >= 0; --c) {  // L^H b = z
            double vr = z[2 * c], vi = z[2 * c + 1];
            for (int m = c + 1; m < r; ++m) {
                // v -= conj(L[m][c]) b[m]
                const double ar = sG[(m * r + c) * 2], ai = -sG[(m * r + c) * 2 + 1];
                vr -= ar * z[2 * m] - ai * z[2 * m + 1];
                vi -= ar * z[2 * m + 1] + ai * z[2 * m];
            }
            const double d = sG[(c * r + c) * 2];
            z[2 * c] = vr / d;
            z[2 * c + 1] = vi / d;
        }
    } else {
        for (int c = 0; c < 2 * r; ++c) z[c] = 0.0;
        atomicOr(status, (unsigned)ST_NOT_SPD_LS);
    }
    for (int l = 0; l < r; ++l) B[(size_t)k * r + l] = make_float2((float)z[2 * l], (float)z[2 * l + 1]);
}

// ---------------------------------------------------------------- D: adjoint, along x

template <int P>
__global__ void __launch_bounds__(256) k_adj_rows(float2 *__restrict__ T, const float2 *__restrict__ B,
                                                   const int32_t *__restrict__ usedrows,
                                                   const int32_t *__restrict__ rfptr, const int32_t *__restrict__ rflist,
                                                   int ny, int r, const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * P;
    extern __shared__ float2 smem[];
    float2 *s_tw = smem;
    float2 *sW = s_tw + NX;
    float2 *tile = sW + RMAXC * RMAXC;
    const int RP = r | 1;
    const int ky = usedrows[blockIdx.x], j = blockIdx.y;
    const size_t n = (size_t)ny * NX;
    load_twiddles(s_tw, g_tw, NX);
    // W_ky = sum over frames sampling row ky of b_k b_k^H
    const int f0 = rfptr[ky], f1 = rfptr[ky + 1];
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        float2 acc = make_float2(0.f, 0.f);
        for (int f = f0; f < f1; ++f) {
            const int k = rflist[f];
            cfma(acc, B[(size_t)k * r + a], cconj(B[(size_t)k * r + b]));
        }
        sW[a * RMAXC + b] = acc;
    }
    float2 *row = T + ((size_t)j * n + (size_t)ky * NX) * r;
    for (int e = threadIdx.x; e < NX * r; e += blockDim.x) {
        const int x = e / r, l = e - x * r;
        tile[x * RP + l] = row[e];
    }
    __syncthreads();
    for (int kx = threadIdx.x; kx < NX; kx += blockDim.x) {
        float2 f[RMAXC];
#pragma unroll
        for (int a = 0; a < RMAXC; ++a) f[a] = (a < r) ? tile[kx * RP + a] : make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < RMAXC; ++b) {
            if (b < r) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < RMAXC; ++a)
                    if (a < r) cfma(acc, f[a], sW[a * RMAXC + b]);
                tile[kx * RP + b] = acc;
            }
        }
    }
    __syncthreads();
    tile_fft<P>(tile, RP, 1, r, s_tw, true, scale);
    __syncthreads();
    for (int e = threadIdx.x; e < NX * r; e += blockDim.x) {
        const int x = e / r, l = e - x * r;
        row[e] = tile[x * RP + l];
    }
}

// ---------------------------------------------------------------- E: adjoint, along y + coil sum

template <int P>
__global__ void __launch_bounds__(256) k_adj_cols(const float2 *__restrict__ T, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, const float2 *__restrict__ Z,
                                                   const float2 *__restrict__ B, float2 *__restrict__ Gout,
                                                   float2 *__restrict__ gpart, unsigned int *counter,
                                                   double *scal, int nx, int r, int q, int nc, double eta_c,
                                                   const float2 *__restrict__ g_tw, float scale) {
    constexpr int NY = 32 * P;
    extern __shared__ float2 smem[];
    float2 *s_tw = smem;
    float2 *tile = s_tw + NY;
    const int RP = r | 1;
    float2 *sS = tile + NY * RP;
    float2 *sB = sS + NY;
    __shared__ float s_c[16], s_s[16];
    __shared__ float2 s_e[16];
    __shared__ int s_cnt;
    __shared__ float2 sA[RMAXC * RMAXC];
    const int x = blockIdx.x;
    const size_t n = (size_t)NY * nx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n1 = brev5(lane);
    load_twiddles(s_tw, g_tw, NY);
    for (int e = threadIdx.x; e < q * r; e += blockDim.x) sB[e] = B[e];
    float2 acc[2][P];
#pragma unroll
    for (int tt = 0; tt < 2; ++tt)
#pragma unroll
        for (int m = 0; m < P; ++m) acc[tt][m] = make_float2(0.f, 0.f);
    for (int j = 0; j < nc; ++j) {
        __syncthreads();
        const float2 *Tj = T + ((size_t)j * n + x) * r;
        for (int e = threadIdx.x; e < NY * r; e += blockDim.x) {
            const int y = e / r, l = e - y * r;
            tile[y * RP + l] = rowused[y] ? Tj[(size_t)y * nx * r + l] : make_float2(0.f, 0.f);
        }
        for (int y = threadIdx.x; y < NY; y += blockDim.x) sS[y] = smaps[(size_t)j * n + (size_t)y * nx + x];
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < 2; ++tt) {
            const int t = warp + 8 * tt;
            if (t < r) {
                float2 v[P];
#pragma unroll
                for (int m = 0; m < P; ++m) v[m] = tile[(n1 + 32 * m) * RP + t];
                warp_fft<P>(v, s_tw, true);
#pragma unroll
                for (int k2 = 0; k2 < P; ++k2) cfmac(acc[tt][k2], sS[k2 + P * lane], cscale(v[k2], scale));
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int tt = 0; tt < 2; ++tt) {
        const int t = warp + 8 * tt;
        if (t < r)
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) tile[(k2 + P * lane) * RP + t] = acc[tt][k2];
    }
    __syncthreads();
    // grad = sum_j conj(d_j) F^H K_j - Z B^H, one thread per pixel of the column
    for (int y = threadIdx.x; y < NY; y += blockDim.x) {
        const size_t i = (size_t)y * nx + x;
        float2 g[RMAXC];
#pragma unroll
        for (int l = 0; l < RMAXC; ++l) g[l] = (l < r) ? tile[y * RP + l] : make_float2(0.f, 0.f);
        const float2 *zr = Z + i * q;
        for (int k = 0; k < q; ++k) {
            const float2 zk = zr[k];
#pragma unroll
            for (int l = 0; l < RMAXC; ++l)
                if (l < r) {
                    const float2 b = sB[k * r + l];
                    // g -= zk * conj(b)
                    g[l].x -= zk.x * b.x + zk.y * b.y;
                    g[l].y -= zk.y * b.x - zk.x * b.y;
                }
        }
#pragma unroll
        for (int l = 0; l < RMAXC; ++l)
            if (l < r) {
                Gout[i * r + l] = g[l];
                tile[y * RP + l] = g[l];
            }
    }
    __syncthreads();
    const int np = r * (r + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        int a, b;
        pair_of(p, r, a, b);
        float2 s = make_float2(0.f, 0.f);
        for (int y = 0; y < NY; ++y) cfmac(s, tile[y * RP + a], tile[y * RP + b]);
        gpart[(size_t)blockIdx.x * np + p] = s;
    }
    if (last_block_arrive(counter)) {
        if (scal[SC_ETASET] == 0.0) {
            // ||grad||_2 = sqrt(lambda_max(grad^H grad)); eta = eta_c / ||grad||_2 (Alg. 2, t = 1)
            for (int p = threadIdx.x; p < np; p += blockDim.x) {
                double re = 0.0, im = 0.0;
                for (int blk = 0; blk < (int)gridDim.x; ++blk) {
                    const float2 v = __ldcg(gpart + (size_t)blk * np + p);
                    re += v.x;
                    im += v.y;
                }
                int a, b;
                pair_of(p, r, a, b);
                sA[a * r + b] = make_float2((float)re, (float)im);
                sA[b * r + a] = make_float2((float)re, (float)-im);
            }
            __syncthreads();
            block_jacobi(sA, r, nullptr, 0, s_c, s_s, s_e, &s_cnt, 30);
            if (threadIdx.x == 0) {
                float lmax = 0.f;
                for (int a = 0; a < r; ++a) lmax = fmaxf(lmax, sA[a * r + a].x);
                const double gn = sqrt((double)lmax);
                scal[SC_GNORM] = gn;
                scal[SC_ETA] = gn > 0.0 ? eta_c / gn : 0.0;
                scal[SC_ETASET] = 1.0;
            }
        }
    }
}

// ---------------------------------------------------------------- F, G, H: GD step and CholeskyQR2

#define QCH 32

// FP64 Cholesky of the r x r Hermitian matrix in sG (re, im pairs), then the
// inverse of R = L^H (upper triangular) into Rinv.  Runs on one thread.
__device__ bool chol_rinv(double *sG, int r, double *Rinv) {
    for (int c = 0; c < r; ++c) {
        double d = sG[(c * r + c) * 2];
        for (int m = 0; m < c; ++m) d -= sG[(c * r + m) * 2] * sG[(c * r + m) * 2] + sG[(c * r + m) * 2 + 1] * sG[(c * r + m) * 2 + 1];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        sG[(c * r + c) * 2] = d;
        sG[(c * r + c) * 2 + 1] = 0.0;
        for (int rr = c + 1; rr < r; ++rr) {
            double vr = sG[(rr * r + c) * 2], vi = sG[(rr * r + c) * 2 + 1];
            for (int m = 0; m < c; ++m) {
                const double ar = sG[(rr * r + m) * 2], ai = sG[(rr * r + m) * 2 + 1];
                const double br = sG[(c * r + m) * 2], bi = sG[(c * r + m) * 2 + 1];
                vr -= ar * br + ai * bi;
                vi -= ai * br - ar * bi;
            }
            sG[(rr * r + c) * 2] = vr / d;
            sG[(rr * r + c) * 2 + 1] = vi / d;
        }
    }
    // Linv (lower) by forward substitution, Rinv = Linv^H
    double Li[RMAXC * RMAXC * 2];
    for (int i = 0; i < r * r * 2; ++i) Li[i] = 0.0;
    for (int i = 0; i < r; ++i) {
        Li[(i * r + i) * 2] = 1.0 / sG[(i * r + i) * 2];
        for (int j = 0; j < i; ++j) {
            double vr = 0.0, vi = 0.0;
            for (int m = j; m < i; ++m) {
                const double ar = sG[(i * r + m) * 2], ai = sG[(i * r + m) * 2 + 1];
                const double br = Li[(m * r + j) * 2], bi = Li[(m * r + j) * 2 + 1];
                vr += ar * br - ai * bi;
                vi += ar * bi + ai * br;
            }
            const double d = sG[(i * r + i) * 2];
            Li[(i * r + j) * 2] = -vr / d;
            Li[(i * r + j) * 2 + 1] = -vi / d;
        }
    }
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            Rinv[(a * r + b) * 2] = Li[(b * r + a) * 2];
            Rinv[(a * r + b) * 2 + 1] = -Li[(b * r + a) * 2 + 1];
        }
    return true;
}

// Reduce the per-block Hermitian partials (np pairs) into sG (FP64).
__device__ void reduce_pairs(const float2 *gpart, int nblk, int r, double *sG) {
    const int np = r * (r + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int blk = 0; blk < nblk; ++blk) {
            const float2 v = __ldcg(gpart + (size_t)blk * np + p);
            re += v.x;
            im += v.y;
        }
        int a, b;
        pair_of(p, r, a, b);
        sG[(a * r + b) * 2] = re;
        sG[(a * r + b) * 2 + 1] = im;
        sG[(b * r + a) * 2] = re;
        sG[(b * r + a) * 2 + 1] = -im;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_gd_gram(const float2 *__restrict__ U, const float2 *__restrict__ Gr,
                                                  float2 *__restrict__ Up, const double *__restrict__ scal,
                                                  float2 *gpart, unsigned int *counter, double *R1inv,
                                                  unsigned int *status, int n, int r, int from_grad) {
    __shared__ float2 s_u[QCH * RMAXC];
    __shared__ double sG[RMAXC * RMAXC * 2];
    const int np = r * (r + 1) / 2;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const float eta = from_grad ? (float)scal[SC_ETA] : 0.f;
    const int p = threadIdx.x;
    int a = 0, b = 0;
    if (p < np) pair_of(p, r, a, b);
    float2 acc = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += QCH) {
        const int cn = min(QCH, i1 - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
            const size_t idx = (size_t)c0 * r + e;
            float2 v;
            if (from_grad) {
                v = csub(U[idx], cscale(Gr[idx], eta));
                Up[idx] = v;
            } else {
                v = Up[idx];
            }
            s_u[e] = v;
        }
        __syncthreads();
        if (p < np)
            for (int ii = 0; ii < cn; ++ii) cfmac(acc, s_u[ii * r + a], s_u[ii * r + b]);
    }
    if (p < np) gpart[(size_t)blockIdx.x * np + p] = acc;
    if (last_block_arrive(counter)) {
        reduce_pairs(gpart, gridDim.x, r, sG);
        if (threadIdx.x == 0) {
            if (!chol_rinv(sG, r, R1inv)) {
                atomicOr(status, (unsigned)ST_NOT_SPD_QR);
                for (int e = 0; e < r * r; ++e) {
                    R1inv[2 * e] = (e / r == e % r) ? 1.0 : 0.0;
                    R1inv[2 * e + 1] = 0.0;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_rinv_gram(const float2 *__restrict__ Up, const double *__restrict__ R1inv,
                                                    float2 *gpart, unsigned int *counter, float2 *M,
                                                    unsigned int *status, int n, int r) {
    __shared__ float2 s_u[QCH * RMAXC];
    __shared__ float2 sR[RMAXC * RMAXC];
    __shared__ double sG[RMAXC * RMAXC * 2];
    __shared__ double sR2[RMAXC * RMAXC * 2];
    const int np = r * (r + 1) / 2;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sR[e] = make_float2((float)R1inv[2 * e], (float)R1inv[2 * e + 1]);
    const int p = threadIdx.x;
    int a = 0, b = 0;
    if (p < np) pair_of(p, r, a, b);
    float2 acc = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += QCH) {
        const int cn = min(QCH, i1 - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
            const int ii = e / r, l = e - ii * r;
            const float2 *u = Up + (size_t)(c0 + ii) * r;
            float2 v = make_float2(0.f, 0.f);
            for (int m = 0; m <= l; ++m) cfma(v, u[m], sR[m * r + l]);
            s_u[e] = v;
        }
        __syncthreads();
        if (p < np)
            for (int ii = 0; ii < cn; ++ii) cfmac(acc, s_u[ii * r + a], s_u[ii * r + b]);
    }
    if (p < np) gpart[(size_t)blockIdx.x * np + p] = acc;
    if (last_block_arrive(counter)) {
        reduce_pairs(gpart, gridDim.x, r, sG);
        if (threadIdx.x == 0) {
            if (!chol_rinv(sG, r, sR2)) {
                atomicOr(status, (unsigned)ST_NOT_SPD_QR);
                for (int e = 0; e < r * r; ++e) {
                    sR2[2 * e] = (e / r == e % r) ? 1.0 : 0.0;
                    sR2[2 * e + 1] = 0.0;
                }
            }
            // M = R1^{-1} R2^{-1}
            for (int i = 0; i < r; ++i)
                for (int jj = 0; jj < r; ++jj) {
                    double vr = 0.0, vi = 0.0;
                    for (int m = 0; m < r; ++m) {
                        const double ar = R1inv[(i * r + m) * 2], ai = R1inv[(i * r + m) * 2 + 1];
                        const double br = sR2[(m * r + jj) * 2], bi = sR2[(m * r + jj) * 2 + 1];
                        vr += ar * br - ai * bi;
                        vi += ar * bi + ai * br;
                    }
                    M[i * r + jj] = make_float2((float)vr, (float)vi);
                }
        }
    }
}

// U_t = U+ M; U_{t-1} kept in Uprev; partials of U_{t-1}^H U_t (for SD) and of
// U_t^H Z (the next iteration's right-hand sides h_k).
#define HMAX 8   // (k, l) pairs per thread: q r <= 256 * 8
__global__ void __launch_bounds__(256) k_apply(float2 *__restrict__ U, float2 *__restrict__ Uprev,
                                                const float2 *__restrict__ Up, const float2 *__restrict__ M,
                                                const float2 *__restrict__ Z, float2 *__restrict__ Hpart,
                                                float2 *gpart, unsigned int *counter, double *scal, int n, int r,
                                                int q, int mode_iter) {
    extern __shared__ float2 smem[];
    float2 *s_up = smem;                 // QCH * r
    float2 *s_new = s_up + QCH * RMAXC;  // QCH * r
    float2 *s_old = s_new + QCH * RMAXC; // QCH * r
    float2 *s_z = s_old + QCH * RMAXC;   // QCH * q
    __shared__ float2 sM[RMAXC * RMAXC];
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sM[e] = M[e];
    float2 cacc = make_float2(0.f, 0.f);
    float2 hacc[HMAX];
#pragma unroll
    for (int u = 0; u < HMAX; ++u) hacc[u] = make_float2(0.f, 0.f);
    const int ca = threadIdx.x / r, cb = threadIdx.x % r;
    const bool cact = threadIdx.x < r * r;
    for (int c0 = i0; c0 < i1; c0 += QCH) {
        const int cn = min(QCH, i1 - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
            s_up[e] = Up[(size_t)c0 * r + e];
            if (mode_iter) s_old[e] = U[(size_t)c0 * r + e];
        }
        for (int e = threadIdx.x; e < cn * q; e += blockDim.x) s_z[e] = Z[(size_t)c0 * q + e];
        __syncthreads();
        for (int e = threadIdx.x; e < cn * r; e += blockDim.x) {
            const int ii = e / r, l = e - ii * r;
            float2 v = make_float2(0.f, 0.f);
            for (int m = 0; m < r; ++m) cfma(v, s_up[ii * r + m], sM[m * r + l]);
            s_new[e] = v;
            U[(size_t)c0 * r + e] = v;
            if (mode_iter) Uprev[(size_t)c0 * r + e] = s_old[e];
        }
        __syncthreads();
        if (mode_iter && cact)
            for (int ii = 0; ii < cn; ++ii) cfmac(cacc, s_old[ii * r + ca], s_new[ii * r + cb]);
#pragma unroll
        for (int u = 0; u < HMAX; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < q * r) {
                const int k = e / r, l = e - k * r;
                for (int ii = 0; ii < cn; ++ii) cfmac(hacc[u], s_new[ii * r + l], s_z[ii * q + k]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < HMAX; ++u) {
        const int e = threadIdx.x + 256 * u;
        if (e < q * r) Hpart[(size_t)blockIdx.x * q * r + e] = hacc[u];
    }
    if (!mode_iter) return;
    if (cact) gpart[(size_t)blockIdx.x * r * r + threadIdx.x] = cacc;
    if (last_block_arrive(counter)) {
        __shared__ double s_red[256];
        double acc = 0.0;
        if (cact) {
            double re = 0.0, im = 0.0;
            for (int blk = 0; blk < (int)gridDim.x; ++blk) {
                const float2 v = __ldcg(gpart + (size_t)blk * r * r + threadIdx.x);
                re += v.x;
                im += v.y;
            }
            acc = re * re + im * im;
        }
        s_red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int e = 0; e < r * r; ++e) s += s_red[e];
            const double sd2 = (double)r - s;
            scal[SC_SD] = sqrt(sd2 > 0.0 ? sd2 : 0.0);
        }
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_qr(lrccs_ctx *c, int from_grad) {
    const int r = c->r;
    prof_begin(c, KID_GD_GRAM);
    k_gd_gram<<<c->nblk, 256, 0, c->stream>>>(c->d_U, c->d_G, c->d_Up, c->d_scal, c->d_gpart,
                                               c->d_counters + CNT_QR1, c->d_R1inv, c->d_status, c->n, r, from_grad);
    prof_end(c, KID_GD_GRAM);
    prof_begin(c, KID_RINV_GRAM);
    k_rinv_gram<<<c->nblk, 256, 0, c->stream>>>(c->d_Up, c->d_R1inv, c->d_gpart, c->d_counters + CNT_QR2, c->d_M,
                                                 c->d_status, c->n, r);
    prof_end(c, KID_RINV_GRAM);
    const size_t smem = (size_t)QCH * (3 * RMAXC + c->q) * sizeof(float2);
    prof_begin(c, KID_APPLY);
    k_apply<<<c->nblk, 256, smem, c->stream>>>(c->d_U, c->d_Uprev, c->d_Up, c->d_M, c->d_Z, c->d_Hpart, c->d_gpart,
                                               c->d_counters + CNT_APPLY, c->d_scal, c->n, r, c->q, from_grad);
    prof_end(c, KID_APPLY);
    return cudaGetLastError();
}

static int fwd_tile_x(int r, int nx) {
    int tx = 1;
    while (tx * 2 * r <= 64 && tx * 2 <= nx) tx *= 2;
    return tx;
}

cudaError_t launch_iteration(lrccs_ctx *c) {
    const int r = c->r, nx = c->nx, ny = c->ny;
    const float sx = (float)(1.0 / sqrt((double)nx));
    const float sy = (float)(1.0 / sqrt((double)ny));
    const int RP = pitch_odd(r);
    const int np = npairs_of(r);
    // A
    {
        const int tx = fwd_tile_x(r, nx);
        const int TP = pitch_odd(tx * r);
        const size_t smem = ((size_t)ny + (size_t)ny * TP) * sizeof(float2);
        dim3 grid(nx / tx, c->nc);
        DISPATCH_P(c->py, {
            prof_begin(c, KID_FWD_COLS);
            k_fwd_cols<P_><<<grid, 256, smem, c->stream>>>(c->d_U, c->d_smaps, c->d_rowused, c->d_T, nx, r, tx,
                                                           c->d_twy, sy);
            prof_end(c, KID_FWD_COLS);
        });
    }
    // B
    {
        const int KG = 256 / np > 0 ? 256 / np : 1;
        const size_t smem = ((size_t)nx + (size_t)nx * RP + (size_t)KG * np) * sizeof(float2);
        const int cpg = (c->nc + c->ncg - 1) / c->ncg;
        dim3 grid(c->n_used, c->ncg);
        DISPATCH_P(c->px, {
            prof_begin(c, KID_FWD_ROWS);
            k_fwd_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_usedrows, c->d_P, ny, r, c->nc, cpg,
                                                           c->d_twx, sx);
            prof_end(c, KID_FWD_ROWS);
        });
    }
    // C
    prof_begin(c, KID_SOLVE);
    k_solve<<<c->q, 64, 0, c->stream>>>(c->d_P, c->d_Hpart, c->d_lineptr, c->d_framerows, ny, r, c->q, c->ncg,
                                        c->nblk, c->d_B, c->d_status);
    prof_end(c, KID_SOLVE);
    // D
    {
        const size_t smem = ((size_t)nx + RMAXC * RMAXC + (size_t)nx * RP) * sizeof(float2);
        dim3 grid(c->n_used, c->nc);
        DISPATCH_P(c->px, {
            prof_begin(c, KID_ADJ_ROWS);
            k_adj_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_B, c->d_usedrows, c->d_rfptr, c->d_rflist,
                                                           ny, r, c->d_twx, sx);
            prof_end(c, KID_ADJ_ROWS);
        });
    }
    // E
    {
        const size_t smem = ((size_t)ny + (size_t)ny * RP + ny + (size_t)c->q * r) * sizeof(float2);
        DISPATCH_P(c->py, {
            prof_begin(c, KID_ADJ_COLS);
            k_adj_cols<P_><<<nx, 256, smem, c->stream>>>(c->d_T, c->d_smaps, c->d_rowused, c->d_Z, c->d_B, c->d_G,
                                                         c->d_gpart, c->d_counters + CNT_GRAD, c->d_scal, nx, r,
                                                         c->q, c->nc, c->prm.eta_c, c->d_twy, sy);
            prof_end(c, KID_ADJ_COLS);
        });
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // F, G, H
    return launch_qr(c, 1);
}

__global__ void k_images(const float2 *__restrict__ Uprev, const float2 *__restrict__ B, float2 *__restrict__ X,
                         int n, int q, int r) {
    const size_t total = (size_t)n * q;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        float2 acc = make_float2(0.f, 0.f);
        for (int l = 0; l < r; ++l) cfma(acc, Uprev[(size_t)i * r + l], B[(size_t)k * r + l]);
        X[e] = acc;
    }
}

cudaError_t launch_images(lrccs_ctx *c, float2 *d_X) {
    prof_begin(c, KID_IMAGES);
    k_images<<<608, 256, 0, c->stream>>>(c->d_Uprev, c->d_B, d_X, c->n, c->q, c->r);
    prof_end(c, KID_IMAGES);
    return cudaGetLastError();
}

#define SET_SMEM(fn) do { cudaError_t e_ = allow_smem(fn, max_smem); if (e_ != cudaSuccess) return e_; } while (0)
#define SET_SMEM_P(fn) \
    SET_SMEM(fn<1>); SET_SMEM(fn<2>); SET_SMEM(fn<3>); SET_SMEM(fn<4>); \
    SET_SMEM(fn<5>); SET_SMEM(fn<6>); SET_SMEM(fn<7>); SET_SMEM(fn<8>)
cudaError_t configure_kernels_iter(int max_smem) {
    SET_SMEM_P(k_fwd_cols);
    SET_SMEM_P(k_fwd_rows);
    SET_SMEM_P(k_adj_rows);
    SET_SMEM_P(k_adj_cols);
    SET_SMEM(k_apply);
    return cudaGetLastError();
}
