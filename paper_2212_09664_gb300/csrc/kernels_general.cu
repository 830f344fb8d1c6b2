// kernels_general.cu -- altGDmin (Alg. 2) with general 2D sampling masks on
// sm_103a: masks whose rows are only partly sampled, such as the pseudo-radial
// golden-angle trajectories gridded onto the Cartesian grid (Sec. V).
//
// With such masks the x-direction transforms no longer cancel.  An iteration
// applies F = F_x F_y to the C r coil images d_j o u_l and keeps the result
// only at the union Omega_u of all frames' samples, stored row by row
// (FU[j][u][l], u = 0 .. n_u - 1 in ascending k-space index).  Linearity gives
//   G_k = (A_k U)^H (A_k U) = sum_{u in Omega_k} P_u,   P_u = sum_j FU_j[u]^H FU_j[u],
//   sum_k A_k^H (A_k U b_k - y_k) b_k^H = sum_j conj(d_j) o F^H [FU_j W] - Z B^H,
//   W_u = sum_{k: u in Omega_k} b_k b_k^H,
// so the iteration still costs C r forward and C r inverse 2D transforms.
//
// Kernels of one iteration (A, F and G are the line path's):
//   A  k_fwd_cols     : F_y(d_j o U) on the rows of Omega_u          -> T[j][ky][x][l]
//   A2 k_fwd_rows     : F_x of each such row, gather of its union points -> FU[j][u][l]
//   B  k_sample_gram  : P_u = sum_j FU_j[u]^H FU_j[u]                 -> Pu[u][pair]
//   C  k_solve_gen    : G_k = sum of P_u over the frame's samples, h_k, Cholesky -> B  (kernels_solve.cu)
//   D  k_sample_w     : FU_j[u] <- FU_j[u] W_u                        -> FU (in place)
//   E  k_adj_rows     : scatter a row's union points, F_x^H           -> T[j][ky][x][l]
//   F  k_adj_cols     : F_y^H and the conj(d_j) coil sum              -> Gk
//   G  k_gdqr         : gradient, GD step, QR                          (kernels_gd.cu)
// and the spectral initialisation's fused pass k_init_gen (Z and X0: direct
// inverse DFT along kx of each frame row's few samples, then the column FFTs).
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

#define RMAXC 16
#define FULLMASK 0xffffffffu

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

// ---------------------------------------------------------------- compaction

// ucnt[i] = number of frames that sample k-space point i.
__global__ void k_union_count(const uint8_t *__restrict__ mask, int q, int n, int32_t *__restrict__ ucnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int k = 0; k < q; ++k) c += mask[(size_t)k * n + i] != 0;
        ucnt[i] = c;
    }
}

// One block of 256 threads per row ky (nx <= 256): exclusive prefix counts of
// the row's union points (uloc, -1 off the union) and of their frame-list
// lengths (floc); the row totals go to urow[ky] and urow[ny + ky].
__global__ void __launch_bounds__(256) k_union_rows(const int32_t *__restrict__ ucnt, int ny, int nx,
                                                     int32_t *__restrict__ uloc, int32_t *__restrict__ floc,
                                                     int32_t *__restrict__ urow) {
    __shared__ int s_a[8], s_b[8];
    const int ky = blockIdx.x, x = threadIdx.x, lane = x & 31, w = x >> 5;
    const int c = x < nx ? ucnt[ky * nx + x] : 0;
    const int f = c > 0 ? 1 : 0;
    int a = f, b = c;   // inclusive warp scans
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ta = __shfl_up_sync(FULLMASK, a, o), tb = __shfl_up_sync(FULLMASK, b, o);
        if (lane >= o) {
            a += ta;
            b += tb;
        }
    }
    if (lane == 31) {
        s_a[w] = a;
        s_b[w] = b;
    }
    __syncthreads();
    int pa = 0, pb = 0;
    for (int v = 0; v < w; ++v) {
        pa += s_a[v];
        pb += s_b[v];
    }
    if (x < nx) {
        uloc[ky * nx + x] = f ? pa + a - 1 : -1;
        floc[ky * nx + x] = pb + b - c;
    }
    if (x == (int)blockDim.x - 1) {
        urow[ky] = pa + a;
        urow[ny + ky] = pb + b;
    }
}

// Row offsets of the union points and of their frame lists (one thread).
__global__ void k_union_scan(const int32_t *__restrict__ urow, int ny, int32_t *__restrict__ uptr,
                             int32_t *__restrict__ ufrow, int32_t *__restrict__ ufptr, int32_t *__restrict__ meta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int a = 0, b = 0;
    for (int ky = 0; ky < ny; ++ky) {
        uptr[ky] = a;
        ufrow[ky] = b;
        a += urow[ky];
        b += urow[ny + ky];
    }
    uptr[ny] = a;
    ufrow[ny] = b;
    ufptr[a] = b;
    meta[MT_NU] = a;
}

// Per union point u (k-space index i): upos[i] = u, uidx[u] = i, and its frames
// in ascending order at uflist[ufptr[u] ..] (a deterministic order, so that
// W_u is summed the same way on every run).
__global__ void k_union_fill(const uint8_t *__restrict__ mask, const int32_t *__restrict__ uloc,
                             const int32_t *__restrict__ floc, const int32_t *__restrict__ uptr,
                             const int32_t *__restrict__ ufrow, int q, int nx, int n, int32_t *__restrict__ upos,
                             int32_t *__restrict__ uidx, int32_t *__restrict__ ufptr, int32_t *__restrict__ uflist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = uloc[i];
        if (l < 0) {
            upos[i] = -1;
            continue;
        }
        const int ky = i / nx;
        const int u = uptr[ky] + l;
        upos[i] = u;
        uidx[u] = i;
        const int f0 = ufrow[ky] + floc[i];
        ufptr[u] = f0;
        int cnt = 0;
        for (int k = 0; k < q; ++k)
            if (mask[(size_t)k * n + i]) uflist[f0 + cnt++] = k;
    }
}

// One warp per (frame k, row ky): the row's samples in ascending kx at
// idx[rowoff ..], and their union indices at fu[rowoff ..].
__global__ void k_fill_general(const uint8_t *__restrict__ mask, const int32_t *__restrict__ rowcnt,
                               const int32_t *__restrict__ rowoff, const int32_t *__restrict__ upos, int q, int ny,
                               int nx, int32_t *__restrict__ idx, int32_t *__restrict__ fu) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= q * ny || rowcnt[w] == 0) return;   // uniform across the warp
    const int k = w / ny, ky = w - k * ny;
    const uint8_t *m = mask + (size_t)k * ny * nx + (size_t)ky * nx;
    int pos = rowoff[w];
    for (int x0 = 0; x0 < nx; x0 += 32) {
        const int x = x0 + lane;
        const bool b = x < nx && m[x] != 0;
        const unsigned bal = __ballot_sync(FULLMASK, b);
        if (b) {
            const int p = pos + __popc(bal & ((1u << lane) - 1u));
            idx[p] = ky * nx + x;
            fu[p] = upos[ky * nx + x];
        }
        pos += __popc(bal);
    }
}

cudaError_t launch_compact_general(lrccs_ctx *c, const uint8_t *d_mask) {
    const int n = c->n, q = c->q, ny = c->ny, nx = c->nx;
    const int blocks = (n + 255) / 256;
    prof_begin(c, KID_UNION);
    k_union_count<<<blocks, 256, 0, c->stream>>>(d_mask, q, n, c->d_ucnt);
    prof_end(c, KID_UNION);
    prof_begin(c, KID_UNION);
    k_union_rows<<<ny, 256, 0, c->stream>>>(c->d_ucnt, ny, nx, c->d_uloc, c->d_floc, c->d_urow);
    prof_end(c, KID_UNION);
    prof_begin(c, KID_UNION);
    k_union_scan<<<1, 32, 0, c->stream>>>(c->d_urow, ny, c->d_uptr, c->d_ufrow, c->d_ufptr, c->d_meta);
    prof_end(c, KID_UNION);
    prof_begin(c, KID_UNION);
    k_union_fill<<<blocks, 256, 0, c->stream>>>(d_mask, c->d_uloc, c->d_floc, c->d_uptr, c->d_ufrow, q, nx, n,
                                                c->d_upos, c->d_uidx, c->d_ufptr, c->d_uflist);
    prof_end(c, KID_UNION);
    prof_begin(c, KID_FILL_GEN);
    k_fill_general<<<(q * ny * 32 + 255) / 256, 256, 0, c->stream>>>(d_mask, c->d_rowcnt, c->d_rowoff, c->d_upos,
                                                                      q, ny, nx, c->d_idx, c->d_fu);
    prof_end(c, KID_FILL_GEN);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init: fused pass

// Z[:, k] = A_k^H y_k and X0[:, k] = A_k^H y_k,tnc / sqrt(m_k mbar) for general
// masks in one pass, block (tile of TXG columns, frame k).  For every coil the
// inverse DFT along kx of each frame row is evaluated directly from the row's
// few samples at the tile's columns (T[ky][x] = sum_s y_s e^{+2 pi i kx_s x / nx}
// / sqrt(nx), plain and truncated), then the column tile is transformed back
// along ky and multiplied by conj(d_j) into the coil sum.  Nothing the size of
// full k-space rows goes through memory.  The block's twiddles
// e^{+2 pi i kx x / nx} (every kx, the tile's x) are tabulated once in shared
// memory; a thread evaluates four columns of one row per pass over its samples.
#define TXG 16
#define IG_STAGE 512    // samples of one coil staged at a time (>= nx: a row always fits)
template <int P>
__global__ void __launch_bounds__(256, 2) k_init_gen(const float2 *__restrict__ y, const int32_t *__restrict__ idx,
                                                     const int32_t *__restrict__ framerows,
                                                     const int32_t *__restrict__ lineptr,
                                                     const int32_t *__restrict__ rowoff,
                                                     const int32_t *__restrict__ rowcnt,
                                                     const int32_t *__restrict__ fpk, const int32_t *__restrict__ mks,
                                                     const float2 *__restrict__ smaps, const double *__restrict__ scal,
                                                     const uint8_t *__restrict__ tflag, float2 *__restrict__ Z,
                                                     float2 *__restrict__ X0, int nx, int q, int nc,
                                                     const float2 *__restrict__ g_twy, const float2 *__restrict__ g_twx,
                                                     float sy, float sx) {
    constexpr int NY = 32 * P;
    constexpr int TP = 2 * TXG + 1;
    constexpr int ACC = (NY * 2 * TXG + 255) / 256;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem;                  // NY * TP
    float2 *s_tw = tile + NY * TP;        // nx * TXG: e^{+2 pi i kx (x0 + xx) / nx} at kx * TXG + xx
    float2 *s_twy = s_tw + nx * TXG;      // NY
    float2 *s_y = s_twy + NY;             // IG_STAGE staged samples of one coil
    int16_t *s_kx = (int16_t *)(s_y + IG_STAGE);
    uint8_t *s_tr = (uint8_t *)(s_kx + IG_STAGE);
    // the frame's rows (the same for every coil): row ky, sample count and
    // first sample, and the row groups whose samples fit the staging area
    __shared__ int s_ky[NY], s_rc[NY], s_ro[NY], s_gb[NY + 1];
    __shared__ int s_ng;
    const int k = blockIdx.y, x0 = blockIdx.x * TXG;
    const int n = NY * nx;
    load_twiddles(s_twy, g_twy, NY);
    for (int e = threadIdx.x; e < nx * TXG; e += blockDim.x) {
        const int kx = e / TXG, xx = e - kx * TXG;
        s_tw[e] = cconj(g_twx[(kx * (x0 + xx)) % nx]);
    }
    const int lp = lineptr[k], L = lineptr[k + 1] - lp;
    const int f0 = fpk[k], mk = mks[k];
    for (int li = threadIdx.x; li < L; li += blockDim.x) {
        const int ky = framerows[lp + li];
        s_ky[li] = ky;
        s_rc[li] = rowcnt[k * NY + ky];
        s_ro[li] = rowoff[k * NY + ky];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ng = 0, tot = 0;
        s_gb[0] = 0;
        for (int li = 0; li < L; ++li) {
            const int c = s_rc[li];
            if (li > 0 && tot + c > IG_STAGE) {
                s_gb[++ng] = li;
                tot = 0;
            }
            tot += c;
        }
        if (L > 0) s_gb[++ng] = L;
        s_ng = ng;
    }
    float2 acc[ACC];
#pragma unroll
    for (int u = 0; u < ACC; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int j = 0; j < nc; ++j) {
        __syncthreads();
        for (int e = threadIdx.x; e < NY * TP; e += blockDim.x) tile[e] = make_float2(0.f, 0.f);
        const int64_t yb = (int64_t)nc * f0 + (int64_t)j * mk;   // sample f0 + s of coil j at y[yb + s]
        // the frame's rows in groups whose samples fit the staging area
        for (int gi = 0; gi < s_ng; ++gi) {
            __syncthreads();
            const int g0 = s_gb[gi], g1 = s_gb[gi + 1];
            const int sbase = s_ro[g0], scnt = s_ro[g1 - 1] + s_rc[g1 - 1] - sbase;
            // stage the group's samples of coil j: value, kx, and the truncation
            // flag (1: |y|^2 > gamma, dropped from the truncated copy)
            for (int e = threadIdx.x; e < scnt; e += blockDim.x) {
                const int s = sbase + e;
                s_y[e] = __ldg(y + yb + (s - f0));
                s_kx[e] = (int16_t)(__ldg(idx + s) % nx);
                s_tr[e] = tflag[yb + (s - f0)];
            }
            __syncthreads();
            // item (row li, column quad cq): columns x0 + 4 cq .. x0 + 4 cq + 3
            for (int e = threadIdx.x; e < (g1 - g0) * (TXG / 4); e += blockDim.x) {
                const int li = g0 + e / (TXG / 4), cq = e % (TXG / 4);
                const int ky = s_ky[li];
                const int off = s_ro[li] - sbase, cnt = s_rc[li];
                float2 vp[4], vt[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) vp[jj] = vt[jj] = make_float2(0.f, 0.f);
                for (int s = off; s < off + cnt; ++s) {
                    const float2 a = s_y[s];
                    const float4 *w4 = (const float4 *)(s_tw + (int)s_kx[s] * TXG + 4 * cq);
                    const float4 wa = w4[0], wb = w4[1];
                    const float2 w[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w), make_float2(wb.x, wb.y),
                                         make_float2(wb.z, wb.w)};
                    const bool keep = s_tr[s] == 0;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        cfma(vp[jj], a, w[jj]);
                        if (keep) cfma(vt[jj], a, w[jj]);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    tile[ky * TP + 2 * (4 * cq + jj)] = cscale(vp[jj], sx);
                    tile[ky * TP + 2 * (4 * cq + jj) + 1] = cscale(vt[jj], sx);
                }
            }
        }
        __syncthreads();
        fft::tile_dft<NY, true>(tile, TP, 2 * TXG, s_twy, sy);
#pragma unroll
        for (int u = 0; u < ACC; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < NY * 2 * TXG) {
                const int yy = e / (2 * TXG), cc = e % (2 * TXG);
                cfmac(acc[u], __ldg(smaps + (size_t)j * n + (size_t)yy * nx + x0 + (cc >> 1)), tile[yy * TP + cc]);
            }
        }
    }
    const double mbar = scal[SC_MBAR];
    const float xs = (mk > 0) ? (float)(1.0 / sqrt((double)mk * mbar)) : 0.f;
#pragma unroll
    for (int u = 0; u < ACC; ++u) {
        const int e = threadIdx.x + 256 * u;
        if (e < NY * 2 * TXG) {
            const int yy = e / (2 * TXG), cc = e % (2 * TXG);
            const size_t i = (size_t)yy * nx + x0 + (cc >> 1);
            if ((cc & 1) == 0) Z[i * q + k] = acc[u];
            else X0[i * q + k] = cscale(acc[u], xs);
        }
    }
}

// The truncation decision of every measured entry, |y|^2 > gamma (FP64 squares,
// as in the line path), once per entry: 1 = dropped from X0.
__global__ void k_trunc_flags(const float2 *__restrict__ y, int64_t count, const double *__restrict__ scal,
                              uint8_t *__restrict__ flag) {
    const double gam = scal[SC_GAMMA];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = abs2_rn(y[e]) > gam ? 1 : 0;
}

cudaError_t launch_init_general(lrccs_ctx *c, const float2 *d_y) {
    const float sx = (float)(1.0 / sqrt((double)c->nx)), sy = (float)(1.0 / sqrt((double)c->ny));
    const size_t smem = ((size_t)c->ny * (2 * TXG + 1) + (size_t)c->nx * TXG + c->ny + IG_STAGE) * sizeof(float2) +
                        (size_t)IG_STAGE * (sizeof(int16_t) + 1);
    prof_begin(c, KID_INIT_GEN);
    k_trunc_flags<<<4 * 152, 256, 0, c->stream>>>(d_y, (int64_t)c->nc * c->total, c->d_scal, c->d_tflag);
    prof_end(c, KID_INIT_GEN);
    dim3 grid(c->nx / TXG, c->q);
    DISPATCH_P(c->py, {
        prof_begin(c, KID_INIT_GEN);
        k_init_gen<P_><<<grid, 256, smem, c->stream>>>(d_y, c->d_idx, c->d_framerows, c->d_lineptr, c->d_rowoff,
                                                       c->d_rowcnt, c->d_fpk, c->d_mks, c->d_smaps, c->d_scal,
                                                       c->d_tflag, c->d_Z, c->d_X0, c->nx, c->q, c->nc, c->d_twy,
                                                       c->d_twx, sy, sx);
        prof_end(c, KID_INIT_GEN);
    });
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A2: forward along x, gather

// Block (row ky of Omega_u, coil group g) transforms the rows of coils g, g +
// CG, ... in turn (double buffered with cp.async): T_j[ky][:][:] (nx x r) is
// transformed along x and its union points written to FU[j][u][:].
template <int PX>
__global__ void __launch_bounds__(256) k_fwd_rows(const float2 *__restrict__ T, const int32_t *__restrict__ usedrows,
                                                   const int32_t *__restrict__ uptr, const int32_t *__restrict__ uidx,
                                                   float2 *__restrict__ FU, int ny, int r, int nc, int nu,
                                                   const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * PX;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile0 = smem, *tile1 = smem + NX * r, *s_tw = tile1 + NX * r;
    __shared__ int s_kx[NX];
    const int ky = usedrows[blockIdx.x], g = blockIdx.y, CG = gridDim.y;
    const size_t plane = (size_t)ny * NX * r;
    const float2 *row0 = T + (size_t)ky * NX * r;
    const int u0 = uptr[ky], cnt = uptr[ky + 1] - u0;
    if (g < nc) stage_row(tile0, row0 + (size_t)g * plane, NX * r, threadIdx.x, blockDim.x);
    cp_async_commit();
    load_twiddles(s_tw, g_tw, NX);
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) s_kx[s] = uidx[u0 + s] - ky * NX;
    const int gl = threadIdx.x % r, gs = threadIdx.x / r, gstep = blockDim.x / r;
    int b = 0;
    for (int j = g; j < nc; j += CG, b ^= 1) {
        float2 *tile = b ? tile1 : tile0;
        if (j + CG < nc) {
            stage_row(b ? tile0 : tile1, row0 + (size_t)(j + CG) * plane, NX * r, threadIdx.x, blockDim.x);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        fft::tile_dft<NX, false>(tile, r, r, s_tw, scale);   // ends with a barrier
        if (gs < gstep) {
            float2 *dst = FU + ((size_t)j * nu + u0) * r;
            for (int s = gs; s < cnt; s += gstep) dst[(size_t)s * r + gl] = tile[s_kx[s] * r + gl];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- B: per-point Gram

// Block of SU = 32 union points: per coil (double buffered) the points' rows
// FU_j[u][:] are staged and every thread adds conj(FU[a]) FU[b] for its
// (point, pair) items; P_u holds the coil sum of the upper triangle.
template <int R>
__global__ void __launch_bounds__(256) k_sample_gram(const float2 *__restrict__ FU, float2 *__restrict__ Pu, int nu,
                                                      int nc) {
    constexpr int np = R * (R + 1) / 2;
    constexpr int SU = 32;
    constexpr int NA = (SU * np + 255) / 256;
    __shared__ __align__(16) float2 s_f[2][SU * R];
    const int u0 = blockIdx.x * SU, cnt = min(SU, nu - u0);
    int ia[NA], ib[NA], io[NA];
    float2 acc[NA];
#pragma unroll
    for (int v = 0; v < NA; ++v) {
        const int o = threadIdx.x + 256 * v;
        acc[v] = make_float2(0.f, 0.f);
        io[v] = -1;
        ia[v] = ib[v] = 0;
        if (o < SU * np) {
            const int s = o / np, p = o - s * np;
            int a, b;
            pair_of(p, R, a, b);
            if (s < cnt) {
                io[v] = o;
                ia[v] = s * R + a;
                ib[v] = s * R + b;
            }
        }
    }
    stage_row(s_f[0], FU + (size_t)u0 * R, cnt * R, threadIdx.x, blockDim.x);
    cp_async_commit();
    for (int j = 0; j < nc; ++j) {
        if (j + 1 < nc) {
            stage_row(s_f[(j + 1) & 1], FU + ((size_t)(j + 1) * nu + u0) * R, cnt * R, threadIdx.x, blockDim.x);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        const float2 *f = s_f[j & 1];
#pragma unroll
        for (int v = 0; v < NA; ++v)
            if (io[v] >= 0) cfmac(acc[v], f[ia[v]], f[ib[v]]);
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < NA; ++v)
        if (io[v] >= 0) Pu[(size_t)u0 * np + io[v]] = acc[v];
}

// ---------------------------------------------------------------- D: times W_u

// Block of SU = 256 / R union points, thread (point su, column wb):
// W_u[:, wb] = sum over the frames k sampling u of b_k conj(b_k[wb]) in
// registers, then for every coil FU_j[u][wb] <- sum_a FU_j[u][a] W_u[a][wb].
template <int R>
__global__ void __launch_bounds__(256) k_sample_w(float2 *__restrict__ FU, const float2 *__restrict__ B,
                                                   const int32_t *__restrict__ ufptr,
                                                   const int32_t *__restrict__ uflist, int nu, int nc, int q) {
    constexpr int SU = 256 / R;
    extern __shared__ __align__(16) float2 smem[];
    float2 *s_f = smem;            // SU * R
    float2 *sB = smem + SU * R;    // q * R
    const int u0 = blockIdx.x * SU, cnt = min(SU, nu - u0);
    const int su = threadIdx.x / R, wb = threadIdx.x - su * R;
    const bool act = su < SU && su < cnt;
    for (int e = threadIdx.x; e < q * R; e += blockDim.x) sB[e] = B[e];
    __syncthreads();
    float2 wcol[R];
#pragma unroll
    for (int a = 0; a < R; ++a) wcol[a] = make_float2(0.f, 0.f);
    if (act) {
        const int u = u0 + su;
        for (int f = ufptr[u]; f < ufptr[u + 1]; ++f) {
            const float2 *bk = sB + uflist[f] * R;
            const float2 bw = cconj(bk[wb]);
#pragma unroll
            for (int a = 0; a < R; ++a) cfma(wcol[a], bk[a], bw);
        }
    }
    for (int j = 0; j < nc; ++j) {
        __syncthreads();
        stage_row(s_f, FU + ((size_t)j * nu + u0) * R, cnt * R, threadIdx.x, blockDim.x);
        cp_async_commit();
        cp_async_wait();
        __syncthreads();
        if (act) {
            float2 o = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < R; ++a) cfma(o, s_f[su * R + a], wcol[a]);
            FU[((size_t)j * nu + u0 + su) * R + wb] = o;
        }
    }
}

// ---------------------------------------------------------------- E: scatter, inverse along x

// Block (row ky of Omega_u, coil group g): for coils g, g + CG, ... the row's
// union points are scattered into a zero row (nx x r), transformed back along
// x, and the full row written to T_j[ky] for the column pass.
template <int PX>
__global__ void __launch_bounds__(256) k_adj_rows(const float2 *__restrict__ FU, const int32_t *__restrict__ usedrows,
                                                   const int32_t *__restrict__ uptr, const int32_t *__restrict__ uidx,
                                                   float2 *__restrict__ T, int ny, int r, int nc, int nu,
                                                   const float2 *__restrict__ g_tw, float scale) {
    constexpr int NX = 32 * PX;
    extern __shared__ __align__(16) float2 smem[];
    float2 *tile = smem, *s_tw = smem + NX * r;
    __shared__ int s_kx[NX];
    const int ky = usedrows[blockIdx.x], g = blockIdx.y, CG = gridDim.y;
    const int u0 = uptr[ky], cnt = uptr[ky + 1] - u0;
    load_twiddles(s_tw, g_tw, NX);
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) s_kx[s] = uidx[u0 + s] - ky * NX;
    const int gl = threadIdx.x % r, gs = threadIdx.x / r, gstep = blockDim.x / r;
    const int half = NX * r / 2;   // float4 pieces of a row (NX is even)
    for (int j = g; j < nc; j += CG) {
        for (int e = threadIdx.x; e < half; e += blockDim.x) ((float4 *)tile)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        if (gs < gstep) {
            const float2 *src = FU + ((size_t)j * nu + u0) * r;
            for (int s = gs; s < cnt; s += gstep) tile[s_kx[s] * r + gl] = src[(size_t)s * r + gl];
        }
        __syncthreads();
        fft::tile_dft<NX, true>(tile, r, r, s_tw, scale);   // ends with a barrier
        float4 *dst = (float4 *)(T + ((size_t)j * ny + ky) * NX * r);
        for (int e = threadIdx.x; e < half; e += blockDim.x) dst[e] = ((const float4 *)tile)[e];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- mean step residual

// y~ = y - A_k zbar for general masks: FU (rank 1) holds F(d_j o zbar) at the
// union points; block (sample chunk, frame k) subtracts it from every coil's
// samples of frame k.
__global__ void k_mean_resid_gen(const float2 *__restrict__ y, const float2 *__restrict__ FU,
                                 const int32_t *__restrict__ fpk, const int32_t *__restrict__ fu, int nc, int nu,
                                 float2 *__restrict__ ytil) {
    const int k = blockIdx.y;
    const int f0 = fpk[k], m = fpk[k + 1] - f0;
    const int64_t base = (int64_t)nc * f0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * m; e += gridDim.x * blockDim.x) {
        const int j = e / m, s = e - j * m;
        const float2 a = y[base + e], b = FU[(size_t)j * nu + fu[f0 + s]];
        ytil[base + e] = make_float2(a.x - b.x, a.y - b.y);
    }
}

// ---------------------------------------------------------------- launchers

static int row_groups(const lrccs_ctx *c) {   // coil groups of the row passes: about 4 coils each, or the plan's
    if (c->plan.row_groups >= 1 && c->plan.row_groups <= 8 && c->plan.row_groups <= c->nc) return c->plan.row_groups;
    const int cg = (c->nc + 3) / 4;
    return cg < 1 ? 1 : (cg > 8 ? 8 : cg);
}

typedef void (*sgram_t)(const float2 *, float2 *, int, int);
typedef void (*sw_t)(float2 *, const float2 *, const int32_t *, const int32_t *, int, int, int);
#define RANK_TABLE(K) {K<1>, K<2>, K<3>, K<4>, K<5>, K<6>, K<7>, K<8>, K<9>, K<10>, K<11>, K<12>, K<13>, K<14>, K<15>, K<16>}
static const sgram_t kSampleGram[RMAXC] = RANK_TABLE(k_sample_gram);
static const sw_t kSampleW[RMAXC] = RANK_TABLE(k_sample_w);

cudaError_t launch_fwd_rows_r(lrccs_ctx *c, int r) {
    const float sx = (float)(1.0 / sqrt((double)c->nx));
    const size_t smem = ((size_t)2 * c->nx * r + c->nx) * sizeof(float2);
    dim3 grid(c->n_used, row_groups(c));
    DISPATCH_P(c->px, {
        prof_begin(c, KID_FWD_ROWS);
        k_fwd_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_usedrows, c->d_uptr, c->d_uidx, c->d_FU, c->ny, r,
                                                       c->nc, c->n_u, c->d_twx, sx);
        prof_end(c, KID_FWD_ROWS);
    });
    return cudaGetLastError();
}

static cudaError_t launch_sample_gram(lrccs_ctx *c) {
    const int r = c->r;
    prof_begin(c, KID_SAMPLE_GRAM);
    kSampleGram[r - 1]<<<(c->n_u + 31) / 32, 256, 0, c->stream>>>(c->d_FU, c->d_Pu, c->n_u, c->nc);
    prof_end(c, KID_SAMPLE_GRAM);
    return cudaGetLastError();
}

cudaError_t launch_sample_w(lrccs_ctx *c) {
    const int r = c->r, su = 256 / r;
    const size_t smem = ((size_t)su * r + (size_t)c->q * r) * sizeof(float2);
    prof_begin(c, KID_SAMPLE_W);
    kSampleW[r - 1]<<<(c->n_u + su - 1) / su, 256, smem, c->stream>>>(c->d_FU, c->d_B, c->d_ufptr, c->d_uflist,
                                                                      c->n_u, c->nc, c->q);
    prof_end(c, KID_SAMPLE_W);
    return cudaGetLastError();
}

cudaError_t launch_adj_rows_r(lrccs_ctx *c, int r) {
    const float sx = (float)(1.0 / sqrt((double)c->nx));
    const size_t smem = ((size_t)c->nx * r + c->nx) * sizeof(float2);
    dim3 grid(c->n_used, row_groups(c));
    DISPATCH_P(c->px, {
        prof_begin(c, KID_ADJ_ROWS);
        k_adj_rows<P_><<<grid, 256, smem, c->stream>>>(c->d_FU, c->d_usedrows, c->d_uptr, c->d_uidx, c->d_T, c->ny, r,
                                                       c->nc, c->n_u, c->d_twx, sx);
        prof_end(c, KID_ADJ_ROWS);
    });
    return cudaGetLastError();
}

cudaError_t launch_fwd_rows(lrccs_ctx *c) { return launch_fwd_rows_r(c, c->r); }
cudaError_t launch_adj_rows(lrccs_ctx *c) { return launch_adj_rows_r(c, c->r); }

cudaError_t launch_iteration_general_front(lrccs_ctx *c) {
    cudaError_t e = launch_fwd_rows(c);
    if (e != cudaSuccess) return e;
    e = launch_sample_gram(c);
    if (e != cudaSuccess) return e;
    return launch_solve(c);
}

cudaError_t launch_iteration_general_back(lrccs_ctx *c) {
    cudaError_t e = launch_sample_w(c);
    if (e != cudaSuccess) return e;
    return launch_adj_rows(c);
}

cudaError_t launch_mean_resid_general(lrccs_ctx *c, const float2 *d_y, float2 *d_ytil) {
    prof_begin(c, KID_MEAN_RESID_GEN);
    k_mean_resid_gen<<<dim3(16, c->q), 256, 0, c->stream>>>(d_y, c->d_FU, c->d_fpk, c->d_fu, c->nc, c->n_u, d_ytil);
    prof_end(c, KID_MEAN_RESID_GEN);
    return cudaGetLastError();
}

#define SET_SMEM(...) do { cudaError_t e_ = allow_smem(__VA_ARGS__, max_smem); if (e_ != cudaSuccess) return e_; } while (0)
cudaError_t configure_kernels_general(int max_smem) {
    SET_SMEM(k_fwd_rows<1>); SET_SMEM(k_fwd_rows<2>); SET_SMEM(k_fwd_rows<3>); SET_SMEM(k_fwd_rows<4>);
    SET_SMEM(k_fwd_rows<5>); SET_SMEM(k_fwd_rows<6>); SET_SMEM(k_fwd_rows<7>); SET_SMEM(k_fwd_rows<8>);
    SET_SMEM(k_adj_rows<1>); SET_SMEM(k_adj_rows<2>); SET_SMEM(k_adj_rows<3>); SET_SMEM(k_adj_rows<4>);
    SET_SMEM(k_adj_rows<5>); SET_SMEM(k_adj_rows<6>); SET_SMEM(k_adj_rows<7>); SET_SMEM(k_adj_rows<8>);
    for (int i = 0; i < RMAXC; ++i) SET_SMEM(kSampleW[i]);
    SET_SMEM(k_init_gen<1>); SET_SMEM(k_init_gen<2>); SET_SMEM(k_init_gen<3>); SET_SMEM(k_init_gen<4>);
    SET_SMEM(k_init_gen<5>); SET_SMEM(k_init_gen<6>); SET_SMEM(k_init_gen<7>); SET_SMEM(k_init_gen<8>);
    return cudaSuccess;
}
