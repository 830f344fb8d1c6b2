// kernels_iter.cu -- the transform kernels of one altGDmin iteration (Alg. 2,
// GDmin loop) on sm_103a.
//
// The iteration uses exact rearrangements of Alg. 2 (linearity only):
//   A_k U = H_k [F(d_j o U)]_j         -> the transforms of U are shared by every frame;
//   (A_k U)^H y_k = U^H Z[:, k]         -> the right-hand side never re-reads y;
//   sum_k A_k^H (A_k U b_k - y_k) b_k^H
//     = sum_j conj(d_j) o F^H [FU_j[i,:] W_i] - Z B^H,   W_i = sum_{k: i in Omega_k} b_k b_k^H.
// With masks that are unions of full k-space rows, H_k keeps whole rows and
// W_i is constant along a row ky.  F = F_y F_x with a unitary F_x, and right
// multiplication by W_ky (acting on the rank index) commutes with F_x, so
//   F_x^H [F_x(T_j[ky, :]) W_ky] = T_j[ky, :] W_ky,   T_j = F_y(d_j o U),
// and by Parseval the row Gram FU^H FU of a row equals T^H T of the same row:
// one iteration needs only the C r column transforms F_y and F_y^H.
//
// Kernels (one launch each per iteration; C is in kernels_solve.cu, I and F in kernels_gd.cu;
// when every sampled row fits one block's shared memory, k_bstep in
// kernels_solve.cu does B, C, D and I in one cooperative launch):
//   A k_fwd_cols  : F_y of d_j o U over column tiles               -> T[j][ky][x][l] (sampled rows)
//   B k_row_gram  : coil-summed row Gram sum_j T_j^H T_j per sampled row -> P[ky] (clusters)
//   C k_solve     : G_k = sum of its rows' P, h_k (sum of k_gdqr's partial rows), Cholesky -> B
//   I k_zb        : Z B^H, on a parallel branch beside D and E          -> ZB
//   D k_row_w     : T_j[ky, :] <- T_j[ky, :] W_ky                    -> T (in place)
//   E k_adj_cols  : F_y^H, conj(d_j) coil sum                      -> Gk
//   F k_gdqr      : grad = Gk - Z B^H, eta (t = 1), U - eta grad and its
//                   Cholesky QR, partial sums of the next h = U^H Z, SD (kernels_gd.cu)
// Tiles are staged into shared memory with cp.async so that each thread keeps
// many loads in flight; the transforms run on the staged tiles (fft.cuh).
#include <cooperative_groups.h>
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched through the runtime)
#include <math.h>
#include <string.h>

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

// ---------------------------------------------------------------- A: forward, along y

// The two tensor maps of a k_fwd_cols launch: U (rows of nx r complex, box
// tx r complex x NY rows) and the coil maps (rows of nx complex over C ny
// rows, box tx complex x NY rows).
struct FwdMaps {
    CUtensorMap u, s;
};

// With TMA, one thread loads the tile of U and of d_j as two tensor copies
// (the tile layouts are the boxes' dense row-major layouts); otherwise every
// thread issues 16-byte cp.async copies.
template <int P, bool TMA>
__global__ void __launch_bounds__(256) k_fwd_cols(const float2 *__restrict__ U, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, float2 *__restrict__ T,
                                                   int nx, int r, int tx, const float2 *__restrict__ g_tw,
                                                   float scale, const __grid_constant__ FwdMaps maps,
                                                   unsigned int *status) {
    constexpr int NY = 32 * P;
    extern __shared__ __align__(128) float2 smem_raw[];
    // 128-byte aligned start (a TMA destination); the launch adds 128 bytes of slack
    float2 *smem = (float2 *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    float2 *tile = smem;                // NY * C
    float2 *sS = tile + NY * tx * r;    // NY * tx
    float2 *s_tw = sS + NY * tx;        // NY
    const int C = tx * r;
    const int x0 = blockIdx.x * tx, j = blockIdx.y;
    const size_t n = (size_t)NY * nx;
    // one copy unit = (row y, 16-byte piece); rows of U are C complex, of d_j tx
    // complex.  Every loop uses a fixed (column, row-step) thread mapping, so no
    // per-element division by the runtime row lengths.
    const int upr = C / 2;
    const int uc = threadIdx.x % upr, uy = threadIdx.x / upr, ustep = blockDim.x / upr;
    if constexpr (TMA) {
        __shared__ __align__(8) uint64_t s_bar;
        if (threadIdx.x == 0) mbar_init(&s_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&s_bar, (unsigned)((NY * C + NY * tx) * sizeof(float2)));
            tma_load_2d(tile, &maps.u, x0 * r * 2, 0, &s_bar);
            tma_load_2d(sS, &maps.s, x0 * 2, j * NY, &s_bar);
        }
        load_twiddles(s_tw, g_tw, NY);
        if (!mbar_wait(&s_bar, 0, 1u << 22) && threadIdx.x == 0) atomicOr(status, (unsigned)ST_TIMEOUT);
        __syncthreads();
    } else {
        const int spr = tx / 2;
        if (uy < ustep)
            for (int y = uy; y < NY; y += ustep)
                cp_async16(tile + y * C + 2 * uc, U + ((size_t)y * nx + x0) * r + 2 * uc);
        {
            const int sc = threadIdx.x % spr, sy = threadIdx.x / spr, sstep = blockDim.x / spr;
            if (sy < sstep)
                for (int y = sy; y < NY; y += sstep)
                    cp_async16(sS + y * tx + 2 * sc, smaps + (size_t)j * n + (size_t)y * nx + x0 + 2 * sc);
        }
        cp_async_commit();
        load_twiddles(s_tw, g_tw, NY);
        cp_async_wait();
        __syncthreads();
    }

    // F_y of d_j o U: the coil multiply happens as pass 1 reads the tile, and
    // pass 2 stores the sampled rows straight to T
    float2 *Tj = T + ((size_t)j * n + x0) * r;
    const size_t rs = (size_t)nx * r;
    fft::tile_dft_io<NY, false>(
        tile, C, C, s_tw, [&](int y, int t) { return cmul(sS[y * tx + t / r], tile[y * C + t]); },
        [&](int t, int ky, float2 v) {
            if (rowused[ky]) Tj[(size_t)ky * rs + t] = cscale(v, scale);
        });
}

// ---------------------------------------------------------------- B: row Gram

// Grid (sampled rows, CG) in clusters of (1, CG): block (ky, g) stages the
// row of coils g, g + CG, ... in turn (double buffered) and accumulates
// sum_j sum_x conj(T_j[ky][x][a]) T_j[ky][x][b] (a <= b) in registers: thread =
// (2 x 2 tile of pairs, x slice).  The slices, then the CG blocks' partials
// (through distributed shared memory), are summed in a fixed order into P[ky].
template <int R>
__global__ void __launch_bounds__(256) k_row_gram(const float2 *__restrict__ T, const int32_t *__restrict__ usedrows,
                                                   float2 *__restrict__ Prow, int ny, int nx, int nc) {
    constexpr int np = R * (R + 1) / 2, tr = (R + 1) / 2, nt = tr * (tr + 1) / 2;
    constexpr int S = 256 / nt;            // x slices per tile
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile0 = smem, *tile1 = smem + nx * R;
    __shared__ float2 s_red[256 * 4];
    __shared__ float2 s_part[np];
    cg::cluster_group cluster = cg::this_cluster();
    const int ky = usedrows[blockIdx.x], g = blockIdx.y, CG = gridDim.y;
    const size_t plane = (size_t)ny * nx * R;
    const float2 *row0 = T + (size_t)ky * nx * R;
    if (g < nc) stage_row(tile0, row0 + (size_t)g * plane, nx * R, threadIdx.x, blockDim.x);
    cp_async_commit();
    const int w = threadIdx.x % nt, sl = threadIdx.x / nt;
    int A, Bt;
    pair_of(w, tr, A, Bt);
    const int x0 = 2 * A, x1 = min(2 * A + 1, R - 1), y0 = 2 * Bt, y1 = min(2 * Bt + 1, R - 1);
    float2 acc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] = make_float2(0.f, 0.f);
    int b = 0;
    for (int j = g; j < nc; j += CG, b ^= 1) {
        const float2 *tile = b ? tile1 : tile0;
        if (j + CG < nc) {
            stage_row(b ? tile0 : tile1, row0 + (size_t)(j + CG) * plane, nx * R, threadIdx.x, blockDim.x);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        if (sl < S) {
#pragma unroll 4
            for (int x = sl; x < nx; x += S) {
                const float2 p0 = tile[x * R + x0], p1 = tile[x * R + x1];
                const float2 q0 = tile[x * R + y0], q1 = tile[x * R + y1];
                cfmac(acc[0], p0, q0);
                cfmac(acc[1], p0, q1);
                cfmac(acc[2], p1, q0);
                cfmac(acc[3], p1, q1);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) s_red[m * 256 + threadIdx.x] = sl < S ? acc[m] : make_float2(0.f, 0.f);
    __syncthreads();
    for (int it = threadIdx.x; it < 4 * nt; it += blockDim.x) {
        const int m = it / nt, ww = it - m * nt;
        int a2, b2;
        pair_of(ww, tr, a2, b2);
        const int a = 2 * a2 + (m >> 1), bq = 2 * b2 + (m & 1);
        if (a < R && bq < R && a <= bq) {
            float2 sum = make_float2(0.f, 0.f);
            for (int ss = 0; ss < S; ++ss) sum = cadd(sum, s_red[m * 256 + ss * nt + ww]);
            s_part[pair_index(a, bq, R)] = sum;
        }
    }
    cluster.sync();
    if (g == 0) {
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            float2 sum = make_float2(0.f, 0.f);
            for (int k = 0; k < CG; ++k) sum = cadd(sum, cluster.map_shared_rank(s_part, k)[p]);
            Prow[(size_t)ky * np + p] = sum;
        }
    }
    cluster.sync();   // no block leaves while its partial may still be read
}

// ---------------------------------------------------------------- D: row times W

// Block (sampled row ky, coil group g): W_ky = sum over the frames k sampling
// row ky of b_k b_k^H (from B staged in shared memory), then for coils g,
// g + CG, ... in turn (double buffered) T_j[ky][x][:] <- T_j[ky][x][:] W_ky in
// place.
template <int R>
__global__ void __launch_bounds__(256) k_row_w(float2 *__restrict__ T, const float2 *__restrict__ B,
                                                const int32_t *__restrict__ usedrows,
                                                const int32_t *__restrict__ rfptr,
                                                const int32_t *__restrict__ rflist, int ny, int nx, int nc, int q) {
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile0 = smem, *tile1 = smem + nx * R;
    float2 *sB = tile1 + nx * R;           // q * R
    __shared__ float2 sW[R * R];
    __shared__ int s_f[256];
    const int ky = usedrows[blockIdx.x], g = blockIdx.y, CG = gridDim.y;
    const size_t plane = (size_t)ny * nx * R;
    float2 *row0 = T + (size_t)ky * nx * R;
    for (int e = threadIdx.x; e < q * R; e += blockDim.x) cp_async8(sB + e, B + e);
    if (g < nc) stage_row(tile0, row0 + (size_t)g * plane, nx * R, threadIdx.x, blockDim.x);
    cp_async_commit();
    const int f0 = rfptr[ky], nf = rfptr[ky + 1] - f0;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) s_f[f] = rflist[f0 + f];
    constexpr int NXG = 256 / R;           // x groups
    const int wb = threadIdx.x % R, xg = threadIdx.x / R;
    float2 wcol[R];
    int b = 0;
    for (int j = g; j < nc; j += CG, b ^= 1) {
        const float2 *tile = b ? tile1 : tile0;
        if (j + CG < nc) {
            stage_row(b ? tile0 : tile1, row0 + (size_t)(j + CG) * plane, nx * R, threadIdx.x, blockDim.x);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        if (j == g) {
            for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
                const int a = e / R, b = e - a * R;
                float2 acc = make_float2(0.f, 0.f);
                for (int f = 0; f < nf; ++f) cfma(acc, sB[s_f[f] * R + a], cconj(sB[s_f[f] * R + b]));
                sW[e] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < R; ++a) wcol[a] = sW[a * R + wb];
        }
        float2 *row = row0 + (size_t)j * plane;
        if (xg < NXG) {   // thread = (output column wb, x group): W_ky[:, wb] in registers
#pragma unroll 2
            for (int x = xg; x < nx; x += NXG) {
                const float2 *fr = tile + x * R;
                float2 o = make_float2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < R; ++a) cfma(o, fr[a], wcol[a]);
                row[x * R + wb] = o;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- E: adjoint, along y + coil sum
// Gk = sum_j conj(d_j) o F_y^H (column x of coil j's row-transformed K_j);
// the - Z B^H term and the Grams are added by k_gdqr (kernels_gd.cu).
//
// Grid (nx, CG) in thread-block clusters of (1, CG): block (x, g) handles
// coils g, g + CG, g + 2 CG, ... of column x and keeps its partial sum in
// registers; the CG partial tiles are then added through distributed shared
// memory in rank order (deterministic), each block writing 1/CG of the column.

// (two chunks: registers capped for two blocks per SM; a third block per SM
// made the one-chunk form slower)
template <int P, int NCH>   // NCH: pass-2 chunks of the 2r transforms (1 or 2)
__global__ void __launch_bounds__(256, NCH == 2 ? 2 : 1) k_adj_cols(const float2 *__restrict__ T, const float2 *__restrict__ smaps,
                                                   const uint8_t *__restrict__ rowused, float2 *__restrict__ Gk,
                                                   int nx, int r, int nc, const float2 *__restrict__ g_tw,
                                                   float scale) {
    constexpr int NY = 32 * P;
    constexpr int R2 = fft::Plan<NY>::R2;
    extern __shared__ __align__(16) float2 smem[];
    // two coils per transform call: tile[y][c r + l], c = 0, 1 (two buffers)
    float2 *tile0 = smem;                 // NY * 2r
    float2 *tile1 = tile0 + NY * 2 * r;
    float2 *sS0 = tile1 + NY * 2 * r;     // 2 NY (two buffers)
    float2 *sS1 = sS0 + 2 * NY;
    float2 *s_tw = sS1 + 2 * NY;          // NY
    cg::cluster_group cluster = cg::this_cluster();
    const int x = blockIdx.x, g = blockIdx.y, CG = gridDim.y;
    const size_t n = (size_t)NY * nx;
    const int cnt = NY * r, r2 = 2 * r;
    // rows that no frame samples are zero-filled
    __shared__ uint8_t s_used[32 * 8];
    for (int y = threadIdx.x; y < NY; y += blockDim.x) s_used[y] = rowused[y];
    // staging map: thread -> rank index l, rows y0, y0 + ystep, ...
    const int sl = threadIdx.x % r, sy0 = threadIdx.x / r, systep = blockDim.x / r;
    // pass-2 accumulators: conj(d_j) F_y^H of every coil of this block, per
    // (chunk, k2) output of tile_dft_acc (a fixed (t, row) per thread)
    float2 acc[NCH][R2];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) acc[ch][k2] = make_float2(0.f, 0.f);
    __syncthreads();
    // coils of this block: g, g + CG, g + 2 CG, ...; step s takes the pair (2s, 2s + 1) of them
    const int mine = g < nc ? (nc - 1 - g) / CG + 1 : 0;
    const int steps = (mine + 1) / 2;
    auto stage = [&](float2 *tile, float2 *sS, int s) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int m = 2 * s + c;
            const int j = g + m * CG;
            const bool live = m < mine;
            const float2 *Tj = T + (size_t)j * n * r + (size_t)x * r;
            if (sy0 < systep)
                for (int y = sy0; y < NY; y += systep) {
                    float2 *dst = tile + y * r2 + c * r + sl;
                    if (live && s_used[y]) cp_async8(dst, Tj + (size_t)y * nx * r + sl);
                    else *dst = make_float2(0.f, 0.f);
                }
            for (int y = threadIdx.x; y < NY; y += blockDim.x) {
                if (live) cp_async8(sS + c * NY + y, smaps + (size_t)j * n + (size_t)y * nx + x);
                else sS[c * NY + y] = make_float2(0.f, 0.f);
            }
        }
        cp_async_commit();
    };
    if (steps > 0) stage(tile0, sS0, 0);
    load_twiddles(s_tw, g_tw, NY);
    for (int s = 0; s < steps; ++s) {
        float2 *tile = (s & 1) ? tile1 : tile0;
        float2 *sS = (s & 1) ? sS1 : sS0;
        if (s + 1 < steps) {
            stage((s & 1) ? tile0 : tile1, (s & 1) ? sS0 : sS1, s + 1);
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        fft::tile_dft_acc<NY, true, NCH>(tile, r2, r2, s_tw, [&](int ch, int k2, int t, int y, float2 v) {
            cfmac(acc[ch][k2], sS[(t >= r ? NY : 0) + y], cscale(v, scale));
        });
        __syncthreads();
    }
    // this block's partial column: the two coil halves added, into tile0[y r + l]
    fft::tile_dft_acc_slots<NY, NCH>(r2, [&](int ch, int k2, int t, int y) { tile1[y * r2 + t] = acc[ch][k2]; });
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int y = e / r, l = e - y * r;
        tile0[e] = cadd(tile1[y * r2 + l], tile1[y * r2 + r + l]);
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

// Columns per k_fwd_cols tile: even, and tx r <= 64 when possible; or the
// context's tuned plan (lrccs_autotune / lrccs_set_plan) when it fits.
bool fwd_tile_ok(int tx, int r, int nx, int ny, int smem_optin) {
    const size_t smem = ((size_t)ny * tx * r + (size_t)ny * tx + ny) * sizeof(float2) + 128;
    return tx >= 2 && (tx & 1) == 0 && nx % tx == 0 && tx * r <= 256 && smem + 256 <= (size_t)smem_optin;
}
static int fwd_tile_x(const lrccs_ctx *c, int r) {
    if (c->plan.fwd_tx && fwd_tile_ok(c->plan.fwd_tx, r, c->nx, c->ny, c->dev_smem_optin)) return c->plan.fwd_tx;
    int tx = 2;
    while (tx * 2 * r <= 64 && tx * 2 <= c->nx) tx *= 2;
    return tx;
}

// Coil groups (cluster size) of k_adj_cols, k_row_gram and k_row_w: groups of
// about 4 coils, at most 8; or the tuned plan's.
static int adj_cluster(const lrccs_ctx *c) {
    if (c->plan.coil_groups >= 1 && c->plan.coil_groups <= 8 && c->plan.coil_groups <= c->nc)
        return c->plan.coil_groups;
    const int cg = (c->nc + 3) / 4;
    return cg < 1 ? 1 : (cg > 8 ? 8 : cg);
}

typedef void (*row_gram_t)(const float2 *, const int32_t *, float2 *, int, int, int);
typedef void (*row_w_t)(float2 *, const float2 *, const int32_t *, const int32_t *, const int32_t *, int, int, int,
                        int);
#define RANK_TABLE(K) {K<1>, K<2>, K<3>, K<4>, K<5>, K<6>, K<7>, K<8>, K<9>, K<10>, K<11>, K<12>, K<13>, K<14>, K<15>, K<16>}
static const row_gram_t kRowGram[RMAXC] = RANK_TABLE(k_row_gram);
static const row_w_t kRowW[RMAXC] = RANK_TABLE(k_row_w);

// One launcher per iteration kernel, at the context's current rank c->r (the
// _on / _to forms take the source or destination and the column count).
// ---------------------------------------------------------------- tensor maps

typedef CUresult (*encode_tiled_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, through the runtime (no link-time
// dependence on libcuda); NULL when unavailable, and the callers then stage
// with cp.async.
static encode_tiled_t tensor_map_encoder() {
    static const encode_tiled_t fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return (encode_tiled_t)p;
    }();
    return fn;
}

// A 2D FP32 tensor map: `outer` rows of `inner` floats, `row_bytes` apart,
// copied in boxes of box_inner x box_outer.  False (nothing encoded) unless
// every TMA rule holds: base and row pitch 16-byte aligned, box edges <= 256
// with an inner extent of a multiple of 16 bytes.
bool encode_map_2d(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                   uint32_t box_inner, uint32_t box_outer) {
    const encode_tiled_t enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15) || (row_bytes & 15) || box_inner < 4 || box_inner > 256 || box_outer < 1 ||
        box_outer > 256 || ((box_inner * 4) & 15) || box_inner > inner || box_outer > outer)
        return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_fwd_cols_on(lrccs_ctx *c, const float2 *src, int r) {
    const int nx = c->nx, ny = c->ny;
    const float sy = (float)(1.0 / sqrt((double)ny));
    const int tx = fwd_tile_x(c, r);
    // 128 bytes of slack: the TMA destination must start 128-byte aligned
    const size_t smem = ((size_t)ny * tx * r + (size_t)ny * tx + ny) * sizeof(float2) + 128;
    dim3 grid(nx / tx, c->nc);
    // the tiles by TMA when both maps encode (x offsets x0 r and x0 are even
    // complex counts: 16-byte aligned, since tx is even)
    FwdMaps maps;
    memset(&maps, 0, sizeof(maps));
    const bool tma = (tx & 1) == 0 &&
                     encode_map_2d(&maps.u, src, (uint64_t)nx * r * 2, (uint64_t)ny, (uint64_t)nx * r * 8,
                                   (uint32_t)(tx * r * 2), (uint32_t)ny) &&
                     encode_map_2d(&maps.s, c->d_smaps, (uint64_t)nx * 2, (uint64_t)c->nc * ny, (uint64_t)nx * 8,
                                   (uint32_t)(tx * 2), (uint32_t)ny);
    DISPATCH_P(c->py, {
        prof_begin(c, KID_FWD_COLS);
        if (tma)
            k_fwd_cols<P_, true><<<grid, 256, smem, c->stream>>>(src, c->d_smaps, c->d_rowused, c->d_T, nx, r, tx,
                                                                 c->d_twy, sy, maps, c->d_status);
        else
            k_fwd_cols<P_, false><<<grid, 256, smem, c->stream>>>(src, c->d_smaps, c->d_rowused, c->d_T, nx, r,
                                                                  tx, c->d_twy, sy, maps, c->d_status);
        prof_end(c, KID_FWD_COLS);
    });
    return cudaSuccess;
}

static cudaError_t launch_row_gram(lrccs_ctx *c) {
    const int r = c->r, nx = c->nx, ny = c->ny;
    const size_t smem = (size_t)2 * nx * r * sizeof(float2);
    const int cgr = adj_cluster(c);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->n_used, cgr, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = cgr;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    prof_begin(c, KID_ROW_GRAM);
    const cudaError_t el = cudaLaunchKernelEx(&cfg, kRowGram[r - 1], (const float2 *)c->d_T,
                                              (const int32_t *)c->d_usedrows, c->d_P, ny, nx, c->nc);
    prof_end(c, KID_ROW_GRAM);
    return el;
}

static void launch_row_w(lrccs_ctx *c) {
    const int r = c->r, nx = c->nx, ny = c->ny;
    const size_t smem = ((size_t)2 * nx * r + (size_t)c->q * r) * sizeof(float2);
    prof_begin(c, KID_ROW_W);
    kRowW[r - 1]<<<dim3(c->n_used, adj_cluster(c)), 256, smem, c->stream>>>(
        c->d_T, c->d_B, c->d_usedrows, c->d_rfptr, c->d_rflist, ny, nx, c->nc, c->q);
    prof_end(c, KID_ROW_W);
}

// coil-summed inverse transform into dst (n x r)
cudaError_t launch_adj_cols_to(lrccs_ctx *c, float2 *dst, int r) {
    const int nx = c->nx, ny = c->ny;
    const float sy = (float)(1.0 / sqrt((double)ny));
    const size_t smem = ((size_t)4 * ny * r + 5 * (size_t)ny) * sizeof(float2);
    const int cg = adj_cluster(c);
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
    // pass-2 chunks of the 2r transforms: 256 / R1 transforms per chunk
    static const int kR1[9] = {0, 4, 8, 12, 8, 10, 12, 14, 16};   // fft::Plan<32 P>::R1
    const int nch = (2 * r + 256 / kR1[c->py] - 1) / (256 / kR1[c->py]);
    if (nch > 2) return cudaErrorInvalidValue;
    cudaError_t el = cudaSuccess;
    DISPATCH_P(c->py, {
        prof_begin(c, KID_ADJ_COLS);
        if (nch == 1)
            el = cudaLaunchKernelEx(&cfg, k_adj_cols<P_, 1>, (const float2 *)c->d_T, (const float2 *)c->d_smaps,
                                    (const uint8_t *)c->d_rowused, dst, nx, r, c->nc, (const float2 *)c->d_twy, sy);
        else
            el = cudaLaunchKernelEx(&cfg, k_adj_cols<P_, 2>, (const float2 *)c->d_T, (const float2 *)c->d_smaps,
                                    (const uint8_t *)c->d_rowused, dst, nx, r, c->nc, (const float2 *)c->d_twy, sy);
        prof_end(c, KID_ADJ_COLS);
    });
    return el;
}

static cudaError_t launch_fwd_cols(lrccs_ctx *c) {
    // the precision forms run the sampled rows' DFT as a tensor-core GEMM
    if (c->dims.precision != LRCCS_PREC_FP32_FFT) return launch_fwd_gemm(c);
    return launch_fwd_cols_on(c, c->d_U, c->r);
}
// the iteration's coil-summed inverse transform goes to the U+ buffer (free during iterations)
static cudaError_t launch_adj_cols(lrccs_ctx *c) { return launch_adj_cols_to(c, c->d_Up, c->r); }

// Z B^H on the context's side stream, forked from (and later joined back
// into) its stream: a parallel branch when the iteration is captured.
static cudaError_t fork_zb(lrccs_ctx *c) {
    cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    if (e != cudaSuccess) return e;
    cudaStream_t main_stream = c->stream;
    c->stream = c->side;
    e = launch_zb(c);
    c->stream = main_stream;
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->side);
    return e;
}
static cudaError_t join_zb(lrccs_ctx *c) { return cudaStreamWaitEvent(c->stream, c->ev_join, 0); }

cudaError_t launch_iteration(lrccs_ctx *c) {
    if (c->r < 1 || c->r > RMAXC) return cudaErrorInvalidValue;
    cudaError_t el = launch_fwd_cols(c);   // A
    if (el != cudaSuccess) return el;
    if (c->general) {                      // 2D masks: x transforms, per-point Grams and W (kernels_general.cu)
        el = launch_iteration_general_front(c);
        if (el != cudaSuccess) return el;
        el = fork_zb(c);                   // I
        if (el != cudaSuccess) return el;
        el = launch_iteration_general_back(c);
        if (el != cudaSuccess) return el;
    } else if (bstep_fused_ok(c)) {
        el = launch_bstep_fused(c);        // B + C + D + I (k_bstep, kernels_solve.cu)
        if (el != cudaSuccess) return el;
        el = launch_adj_cols(c);           // E
        if (el != cudaSuccess) return el;
        return launch_gdqr(c, 1);          // F
    } else {
        el = launch_row_gram(c);           // B
        if (el != cudaSuccess) return el;
        launch_solve(c);                   // C
        el = fork_zb(c);                   // I
        if (el != cudaSuccess) return el;
        launch_row_w(c);                   // D
    }
    el = launch_adj_cols(c);               // E
    if (el != cudaSuccess) return el;
    el = join_zb(c);
    if (el != cudaSuccess) return el;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // F: gradient, GD step and Cholesky QR (one cooperative launch)
    return launch_gdqr(c, 1);
}

// The iteration's forward transform alone (FP32 FFT or, for the precision
// forms, the tensor-core GEMM): d_T <- F_y(d_j o U) on the sampled rows.
cudaError_t launch_forward(lrccs_ctx *c) {
    if (c->r < 1 || c->r > RMAXC) return cudaErrorInvalidValue;
    cudaError_t el = launch_fwd_cols(c);
    if (el != cudaSuccess) return el;
    return cudaGetLastError();
}

// The B-step alone at the current U (the partial sums of U^H Z left by the
// k_gdqr launch that formed U): forward transforms, Grams and the per-frame
// solves.
cudaError_t launch_bstep(lrccs_ctx *c) {
    if (c->r < 1 || c->r > RMAXC) return cudaErrorInvalidValue;
    cudaError_t el = launch_fwd_cols(c);
    if (el != cudaSuccess) return el;
    if (c->general) return launch_iteration_general_front(c);
    el = launch_row_gram(c);
    if (el != cudaSuccess) return el;
    return launch_solve(c);
}

// The normal operator of the stacked A = [A_1; ...; A_q] with B = 1 (q x 1):
// d_Up <- sum_j conj(d_j) o F^H[c o F(d_j o u)], u = d_U (n x 1), c_i the
// number of frames that sample k-space row i (W_i of the gradient with r = 1).
cudaError_t launch_normal_op(lrccs_ctx *c) {
    if (c->r != 1) return cudaErrorInvalidValue;
    cudaError_t el = launch_fwd_cols(c);
    if (el != cudaSuccess) return el;
    if (c->general) {   // W_u = number of frames sampling point u
        el = launch_fwd_rows(c);
        if (el == cudaSuccess) el = launch_sample_w(c);
        if (el == cudaSuccess) el = launch_adj_rows(c);
        if (el != cudaSuccess) return el;
    } else {
        launch_row_w(c);
    }
    el = launch_adj_cols(c);
    if (el != cudaSuccess) return el;
    return cudaGetLastError();
}

// d_T <- F_y(d_j o U) on the sampled rows (the first step of an iteration);
// with general masks also d_FU <- F(d_j o U) at the union points.
cudaError_t launch_fwd_only(lrccs_ctx *c) {
    if (c->r < 1 || c->r > RMAXC) return cudaErrorInvalidValue;
    cudaError_t el = launch_fwd_cols(c);
    if (el != cudaSuccess) return el;
    if (c->general) {
        el = launch_fwd_rows(c);
        if (el != cudaSuccess) return el;
    }
    return cudaGetLastError();
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
    SET_SMEM(k_fwd_cols<1, false>); SET_SMEM(k_fwd_cols<2, false>); SET_SMEM(k_fwd_cols<3, false>);
    SET_SMEM(k_fwd_cols<4, false>); SET_SMEM(k_fwd_cols<5, false>); SET_SMEM(k_fwd_cols<6, false>);
    SET_SMEM(k_fwd_cols<7, false>); SET_SMEM(k_fwd_cols<8, false>);
    SET_SMEM(k_fwd_cols<1, true>); SET_SMEM(k_fwd_cols<2, true>); SET_SMEM(k_fwd_cols<3, true>);
    SET_SMEM(k_fwd_cols<4, true>); SET_SMEM(k_fwd_cols<5, true>); SET_SMEM(k_fwd_cols<6, true>);
    SET_SMEM(k_fwd_cols<7, true>); SET_SMEM(k_fwd_cols<8, true>);
    for (int i = 0; i < RMAXC; ++i) {
        SET_SMEM(kRowGram[i]);
        SET_SMEM(kRowW[i]);
    }
    SET_SMEM(k_adj_cols<1, 1>); SET_SMEM(k_adj_cols<2, 1>); SET_SMEM(k_adj_cols<3, 1>); SET_SMEM(k_adj_cols<4, 1>);
    SET_SMEM(k_adj_cols<5, 1>); SET_SMEM(k_adj_cols<6, 1>); SET_SMEM(k_adj_cols<7, 1>); SET_SMEM(k_adj_cols<8, 1>);
    SET_SMEM(k_adj_cols<1, 2>); SET_SMEM(k_adj_cols<2, 2>); SET_SMEM(k_adj_cols<3, 2>); SET_SMEM(k_adj_cols<4, 2>);
    SET_SMEM(k_adj_cols<5, 2>); SET_SMEM(k_adj_cols<6, 2>); SET_SMEM(k_adj_cols<7, 2>); SET_SMEM(k_adj_cols<8, 2>);
    return cudaSuccess;
}
