// kernels_iter.cu -- the transform kernels of one altGDmin iteration (Alg. 2,
// GDmin loop) on sm_103a.
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
// Kernels (one launch each per iteration; C is in kernels_solve.cu, F in kernels_gd.cu):
//   A k_fwd_cols  : F_y of d_j o U over column tiles               -> T[j][ky][x][l]
//   B k_fwd_rows  : F_x of every sampled row of one coil, row Gram -> FU (in place), P[j][ky]
//   C k_solve     : G_k = sum of its rows' P, h_k, Cholesky         -> B
//   D k_adj_rows  : K = FU W_ky, F_x^H                              -> T (in place)
//   E k_adj_cols  : F_y^H, conj(d_j) coil sum                      -> Gk
//   F k_gdqr      : grad = Gk - Z B^H, eta (t = 1), U - eta grad and its
//                   CholeskyQR2, h = U^H Z, SD                      (kernels_gd.cu)
// Tiles are staged into shared memory with cp.async so that each thread keeps
// many loads in flight; the transforms run on the staged tiles (fft.cuh).
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

#define DISPATCH_P(PV, ...)                                            \
    switch (PV) {                                                      \
        case 1: { constexpr int P_ = 1; __VA_ARGS__; } break;          \
        case 2: { constexpr int P_ = 2; __VA_ARGS__; } break;          \
        case 3: { constexpr int P_ = 3; __VA_ARGS__; } break;          \
        case 4: { constexpr int P_ = 4; __VA_ARGS__; } break;          \
        case 5: { constexpr int P_ = 5; __VA_ARGS__; } break;          \
        case 6: { constexpr int P_ = 6; __VA_ARGS__; } break;          \
        case 7: { constexpr int P_ = 7; __VA_ARGS__; } break;          \
        case 8: { constexpr int P_ = 8; __VA_ARGS__; } break;          \
        default: return cudaErrorInvalidValue;                         \
    }

#define RMAXC 16   // compile-time bound on the rank

int npairs_of(int r) { return r * (r + 1) / 2; }

// Stage `count` complex64 values from global `src` into shared `dst`, 16 bytes
// per copy when both are 16-byte aligned and count is even, else 8 bytes.
LRCCS_DEV void stage_row(float2 *dst, const float2 *src, int count, int tid, int nthr) {
    if (((((uintptr_t)src) | smem_u32(dst)) & 15) == 0 && (count & 1) == 0) {
        for (int e = tid; e < count / 2; e += nthr) cp_async16(dst + 2 * e, src + 2 * e);
    } else {
        for (int e = tid; e < count; e += nthr) cp_async8(dst + e, src + e);
    }
}

// ---------------------------------------------------------------- A: forward, along y

template <int P>
__global__ void __launch_bounds__(256) k_fwd_cols(const float2 *__restrict__ U, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, float2 *__restrict__ T,
                                                   int nx, int r, int tx, const float2 *__restrict__ g_tw,
                                                   float scale) {
    constexpr int NY = 32 * P;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem;                // NY * C
    float2 *sS = tile + NY * tx * r;    // NY * tx
    float2 *s_tw = sS + NY * tx;        // NY
    const int C = tx * r;
    const int x0 = blockIdx.x * tx, j = blockIdx.y;
    const size_t n = (size_t)NY * nx;
    // one copy unit = (row y, 16-byte piece); rows of U are C complex, of d_j tx complex
    const int upr = C / 2, spr = tx / 2;
    for (int e = threadIdx.x; e < NY * upr; e += blockDim.x) {
        const int y = e / upr, c2 = e - y * upr;
        cp_async16(tile + y * C + 2 * c2, U + ((size_t)y * nx + x0) * r + 2 * c2);
    }
    for (int e = threadIdx.x; e < NY * spr; e += blockDim.x) {
        const int y = e / spr, c2 = e - y * spr;
        cp_async16(sS + y * tx + 2 * c2, smaps + (size_t)j * n + (size_t)y * nx + x0 + 2 * c2);
    }
    cp_async_commit();
    load_twiddles(s_tw, g_tw, NY);
    cp_async_wait();
    __syncthreads();
    for (int e = threadIdx.x; e < NY * C; e += blockDim.x) {
        const int y = e / C, c = e - y * C;
        tile[e] = cmul(sS[y * tx + c / r], tile[e]);
    }
    __syncthreads();
    fft::tile_dft<NY, false>(tile, C, C, s_tw, scale);
    float2 *Tj = T + ((size_t)j * n + x0) * r;
    for (int e = threadIdx.x; e < NY * upr; e += blockDim.x) {
        const int ky = e / upr, c2 = e - ky * upr;
        if (rowused[ky])
            *(float4 *)(Tj + (size_t)ky * nx * r + 2 * c2) = *(const float4 *)(tile + ky * C + 2 * c2);
    }
}

// ---------------------------------------------------------------- B: forward, along x + row Gram

// The last of a row's nc blocks to finish also sums the row's coil partials
// (in coil order) into Ppart[nc][ky], the coil-summed row Gram used by k_solve.
template <int P>
__global__ void __launch_bounds__(256) k_fwd_rows(float2 *__restrict__ T, const int32_t *__restrict__ usedrows,
                                                   float2 *__restrict__ Ppart, unsigned int *__restrict__ arrive,
                                                   int ny, int r, const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * P;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem;               // NX * r
    float2 *s_tw = tile + NX * r;      // NX
    float2 *s_red = s_tw + NX;         // KG * np
    const int ky = usedrows[blockIdx.x], j = blockIdx.y;
    const size_t n = (size_t)ny * NX;
    float2 *row = T + ((size_t)j * n + (size_t)ky * NX) * r;
    stage_row(tile, row, NX * r, threadIdx.x, blockDim.x);
    cp_async_commit();
    load_twiddles(s_tw, g_tw, NX);
    const int np = r * (r + 1) / 2;
    const int KG = max(1, (int)blockDim.x / np);
    const int p = threadIdx.x % np, kg = threadIdx.x / np;
    const bool active = kg < KG;
    int a = 0, b = 0;
    pair_of(p, r, a, b);
    cp_async_wait();
    __syncthreads();
    fft::tile_dft<NX, false>(tile, r, r, s_tw, scale);
    for (int e = threadIdx.x; e < NX * r / 2; e += blockDim.x)
        ((float4 *)row)[e] = ((const float4 *)tile)[e];
    float2 acc = make_float2(0.f, 0.f);
    if (active)
        for (int kx = kg; kx < NX; kx += KG) cfmac(acc, tile[kx * r + a], tile[kx * r + b]);
    if (active) s_red[kg * np + p] = acc;
    __syncthreads();
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < KG; ++g) s = cadd(s, s_red[g * np + pp]);
        Ppart[((size_t)j * ny + ky) * np + pp] = s;
    }
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {   // the fence after the barrier releases the whole block's writes
        __threadfence();
        const unsigned int prev = atomicAdd(arrive + ky, 1u);
        s_last = prev == gridDim.y - 1;
        if (s_last) arrive[ky] = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nc = gridDim.y;
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = 0; g < nc; ++g) s = cadd(s, __ldcg(Ppart + ((size_t)g * ny + ky) * np + pp));
        Ppart[((size_t)nc * ny + ky) * np + pp] = s;
    }
}

// ---------------------------------------------------------------- D: adjoint, along x

template <int P>
__global__ void __launch_bounds__(256) k_adj_rows(float2 *__restrict__ T, const float2 *__restrict__ B,
                                                   const int32_t *__restrict__ usedrows,
                                                   const int32_t *__restrict__ rfptr, const int32_t *__restrict__ rflist,
                                                   int ny, int r, const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * P;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem;                 // NX * r
    float2 *s_tw = tile + NX * r;        // NX
    float2 *sW = s_tw + NX;              // RMAXC * RMAXC
    const int ky = usedrows[blockIdx.x], j = blockIdx.y;
    const size_t n = (size_t)ny * NX;
    float2 *row = T + ((size_t)j * n + (size_t)ky * NX) * r;
    stage_row(tile, row, NX * r, threadIdx.x, blockDim.x);
    cp_async_commit();
    load_twiddles(s_tw, g_tw, NX);
    // W_ky = sum over the frames sampling row ky of b_k b_k^H (while the row arrives)
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
    cp_async_wait();
    __syncthreads();
    for (int kx = threadIdx.x; kx < NX; kx += blockDim.x) {
        float2 f[RMAXC];
#pragma unroll
        for (int a = 0; a < RMAXC; ++a) f[a] = (a < r) ? tile[kx * r + a] : make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < RMAXC; ++b) {
            if (b < r) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < RMAXC; ++a)
                    if (a < r) cfma(acc, f[a], sW[a * RMAXC + b]);
                tile[kx * r + b] = acc;
            }
        }
    }
    __syncthreads();
    fft::tile_dft<NX, true>(tile, r, r, s_tw, scale);
    for (int e = threadIdx.x; e < NX * r / 2; e += blockDim.x)
        ((float4 *)row)[e] = ((const float4 *)tile)[e];
}

// ---------------------------------------------------------------- E: adjoint, along y + coil sum
// Gk = sum_j conj(d_j) o F_y^H (column x of coil j's row-transformed K_j);
// the - Z B^H term and the Grams are added by k_gdqr (kernels_gd.cu).
//
// Grid (nx, CG) in thread-block clusters of (1, CG): block (x, g) handles
// coils g, g + CG, g + 2 CG, ... of column x and keeps its partial sum in
// registers; the CG partial tiles are then added through distributed shared
// memory in rank order (deterministic), each block writing 1/CG of the column.

template <int P, int EA>   // EA: tile elements per thread, NY r <= 256 EA
__global__ void __launch_bounds__(256) k_adj_cols(const float2 *__restrict__ T, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, float2 *__restrict__ Gk,
                                                   int nx, int r, int nc, const float2 *__restrict__ g_tw,
                                                   float scale) {
    constexpr int NY = 32 * P;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile0 = smem;                 // NY * r (two buffers)
    float2 *tile1 = tile0 + NY * r;
    float2 *sS0 = tile1 + NY * r;         // NY (two buffers)
    float2 *sS1 = sS0 + NY;
    float2 *s_tw = sS1 + NY;              // NY
    cg::cluster_group cluster = cg::this_cluster();
    const int x = blockIdx.x, g = blockIdx.y, CG = gridDim.y;
    const size_t n = (size_t)NY * nx;
    const int cnt = NY * r;
    // this thread's tile elements e = tid + 256 u: global offset of (y, l) in a
    // coil plane, or -1 for rows no frame samples
    int goff[EA];
#pragma unroll
    for (int u = 0; u < EA; ++u) {
        const int e = threadIdx.x + 256 * u;
        goff[u] = -2;
        if (e < cnt) {
            const int y = e / r, l = e - y * r;
            goff[u] = rowused[y] ? (int)(((size_t)y * nx + x) * r + l) : -1;
        }
    }
    auto stage = [&](float2 *tile, float2 *sS, int j) {
        const float2 *Tj = T + (size_t)j * n * r;
#pragma unroll
        for (int u = 0; u < EA; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (goff[u] >= 0) cp_async8(tile + e, Tj + goff[u]);
            else if (goff[u] == -1) tile[e] = make_float2(0.f, 0.f);
        }
        for (int y = threadIdx.x; y < NY; y += blockDim.x) cp_async8(sS + y, smaps + (size_t)j * n + (size_t)y * nx + x);
        cp_async_commit();
    };
    float2 acc[EA];
#pragma unroll
    for (int u = 0; u < EA; ++u) acc[u] = make_float2(0.f, 0.f);
    if (g < nc) stage(tile0, sS0, g);
    load_twiddles(s_tw, g_tw, NY);
    int b = 0;
    for (int j = g; j < nc; j += CG, b ^= 1) {
        float2 *tile = b ? tile1 : tile0;
        float2 *sS = b ? sS1 : sS0;
        if (j + CG < nc) {
            stage(b ? tile0 : tile1, b ? sS0 : sS1, j + CG);
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        fft::tile_dft<NY, true>(tile, r, r, s_tw, scale);
#pragma unroll
        for (int u = 0; u < EA; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < cnt) cfmac(acc[u], sS[e / r], tile[e]);
        }
        __syncthreads();
    }
    // partial tile of this block into its own tile0, then the cluster-wide sum
#pragma unroll
    for (int u = 0; u < EA; ++u) {
        const int e = threadIdx.x + 256 * u;
        if (e < cnt) tile0[e] = acc[u];
    }
    cluster.sync();
    const int per = (cnt + CG - 1) / CG;
    const int e0 = g * per, e1 = min(cnt, e0 + per);
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 sum = make_float2(0.f, 0.f);
        for (int k = 0; k < CG; ++k) sum = cadd(sum, cluster.map_shared_rank(tile0, k)[e]);
        const int y = e / r, l = e - y * r;
        Gk[((size_t)y * nx + x) * r + l] = sum;
    }
    cluster.sync();   // no block leaves while its tile may still be read
}

// ---------------------------------------------------------------- launchers

// Blocks per cluster of k_adj_cols: groups of about 4 coils, at most 8 blocks.
static int adj_cluster(int nc) {
    const int cg = (nc + 3) / 4;
    return cg < 1 ? 1 : (cg > 8 ? 8 : cg);
}

// Columns per k_fwd_cols tile: even, and tx r <= 64 when possible.
static int fwd_tile_x(int r, int nx) {
    int tx = 2;
    while (tx * 2 * r <= 64 && tx * 2 <= nx) tx *= 2;
    return tx;
}

cudaError_t launch_iteration(lrccs_ctx *c) {
    const int r = c->r, nx = c->nx, ny = c->ny;
    const float sx = (float)(1.0 / sqrt((double)nx));
    const float sy = (float)(1.0 / sqrt((double)ny));
    const int np = npairs_of(r);
    // A
    {
        const int tx = fwd_tile_x(r, nx);
        const size_t smem = ((size_t)ny * tx * r + (size_t)ny * tx + ny) * sizeof(float2);
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
        const size_t smem = ((size_t)nx * r + nx + (size_t)KG * np) * sizeof(float2);
        dim3 grid(c->n_used, c->nc);
        DISPATCH_P(c->px, {
            prof_begin(c, KID_FWD_ROWS);
            k_fwd_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_usedrows, c->d_P, c->d_rowarrive, ny, r,
                                                           c->d_twx, sx);
            prof_end(c, KID_FWD_ROWS);
        });
    }
    // C
    launch_solve(c);
    // D
    {
        const size_t smem = ((size_t)nx * r + nx + RMAXC * RMAXC) * sizeof(float2);
        dim3 grid(c->n_used, c->nc);
        DISPATCH_P(c->px, {
            prof_begin(c, KID_ADJ_ROWS);
            k_adj_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_B, c->d_usedrows, c->d_rfptr, c->d_rflist,
                                                           ny, r, c->d_twx, sx);
            prof_end(c, KID_ADJ_ROWS);
        });
    }
    // E: coil-summed inverse transform into the U+ buffer (free during iterations)
    {
        const size_t smem = ((size_t)2 * ny * r + 3 * (size_t)ny) * sizeof(float2);
        const int cg = adj_cluster(c->nc);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nx, cg, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = cg;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const bool small = ny * r <= 256 * 8;
        cudaError_t el = cudaSuccess;
        DISPATCH_P(c->py, {
            prof_begin(c, KID_ADJ_COLS);
            if (small)
                el = cudaLaunchKernelEx(&cfg, k_adj_cols<P_, 8>, (const float2 *)c->d_T, (const float2 *)c->d_smaps,
                                        (const uint8_t *)c->d_rowused, c->d_Up, nx, r, c->nc, (const float2 *)c->d_twy, sy);
            else
                el = cudaLaunchKernelEx(&cfg, k_adj_cols<P_, 16>, (const float2 *)c->d_T, (const float2 *)c->d_smaps,
                                        (const uint8_t *)c->d_rowused, c->d_Up, nx, r, c->nc, (const float2 *)c->d_twy, sy);
            prof_end(c, KID_ADJ_COLS);
        });
        if (el != cudaSuccess) return el;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // F: gradient, GD step and CholeskyQR2 (one cooperative launch)
    return launch_gdqr(c, 1);
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

#define SET_SMEM(...) do { cudaError_t e_ = allow_smem(__VA_ARGS__, max_smem); if (e_ != cudaSuccess) return e_; } while (0)
#define SET_SMEM_P(fn) \
    SET_SMEM(fn<1>); SET_SMEM(fn<2>); SET_SMEM(fn<3>); SET_SMEM(fn<4>); \
    SET_SMEM(fn<5>); SET_SMEM(fn<6>); SET_SMEM(fn<7>); SET_SMEM(fn<8>)
cudaError_t configure_kernels_iter(int max_smem) {
    SET_SMEM_P(k_fwd_cols);
    SET_SMEM_P(k_fwd_rows);
    SET_SMEM_P(k_adj_rows);
    SET_SMEM(k_adj_cols<1, 8>); SET_SMEM(k_adj_cols<2, 8>); SET_SMEM(k_adj_cols<3, 8>); SET_SMEM(k_adj_cols<4, 8>);
    SET_SMEM(k_adj_cols<5, 8>); SET_SMEM(k_adj_cols<6, 8>); SET_SMEM(k_adj_cols<7, 8>); SET_SMEM(k_adj_cols<8, 8>);
    SET_SMEM(k_adj_cols<1, 16>); SET_SMEM(k_adj_cols<2, 16>); SET_SMEM(k_adj_cols<3, 16>); SET_SMEM(k_adj_cols<4, 16>);
    SET_SMEM(k_adj_cols<5, 16>); SET_SMEM(k_adj_cols<6, 16>); SET_SMEM(k_adj_cols<7, 16>); SET_SMEM(k_adj_cols<8, 16>);
    return cudaSuccess;
}
