// kernels_init.cu -- spectral initialisation of auto-altGDmin (Alg. 2, init)
// on sm_103a: mask compaction, gamma, Z = [A_k^H y_k], truncated X0, the q x q
// Gram X0^H X0 with a Jacobi eigensolver, and U_0 = X0 V_r Sigma_r^{-1}.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

// ---------------------------------------------------------------- twiddles

__global__ void k_twiddles(float2 *tw, int N) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)N, &s, &c);  // exp(-2 pi i t / N)
        tw[t] = make_float2((float)c, (float)s);
    }
}

cudaError_t launch_twiddles(float2 *tw, int N, cudaStream_t s) {
    k_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- mask compaction
// Sampling H_k (Sec. II-A) given as a q x n bitmap.  This build accepts masks
// whose every row ky is either fully sampled or empty (1D Cartesian lines).

__global__ void k_rowcount(const uint8_t *__restrict__ mask, int rows, int nx, int32_t *rowcnt) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows) return;
    const uint8_t *m = mask + (size_t)w * nx;
    int c = 0;
    for (int x = lane; x < nx; x += 32) c += (m[x] != 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) rowcnt[w] = c;
}

// Per-frame and per-row structure of the masks from the per-(frame, row)
// sample counts.  Rows of a frame with at least one sample are the frame's
// "frame rows" (its lines, for 1D Cartesian masks): lineptr / framerows /
// framek / rowidx.  Also the frames' sample counts m_k and offsets fpk (checked
// against the caller's frame_ptr), each (frame, row)'s first sample rowoff, the
// rows sampled by some frame, and meta[MT_GENERAL] = 1 when some row is only
// partly sampled (a general 2D mask).
__global__ void k_structure(const int32_t *__restrict__ rowcnt, const int64_t *__restrict__ fp_user,
                            int q, int ny, int nx, int32_t *rowidx, int32_t *framerows, int32_t *framek,
                            int32_t *lineptr, int32_t *rfptr, int32_t *rflist, int32_t *usedrows,
                            uint8_t *rowused, int32_t *mks, int32_t *fpk, int32_t *rowoff, int32_t *meta,
                            unsigned int *status, double *scal) {
    __shared__ int s_lines[129];
    __shared__ int s_m[129];
    __shared__ int s_fp[130];
    __shared__ int s_rf[257];
    __shared__ int s_partial;
    const int tid = threadIdx.x;
    if (tid == 0) s_partial = 0;
    __syncthreads();
    for (int k = tid; k < q; k += blockDim.x) {
        int L = 0, m = 0, part = 0;
        for (int ky = 0; ky < ny; ++ky) {
            const int c = rowcnt[k * ny + ky];
            L += c > 0;
            m += c;
            part |= (c != 0 && c != nx);
        }
        s_lines[k] = L;
        s_m[k] = m;
        if (part) s_partial = 1;
    }
    for (int ky = tid; ky < ny; ky += blockDim.x) {
        int c = 0;
        for (int k = 0; k < q; ++k) c += (rowcnt[k * ny + ky] > 0);
        s_rf[ky] = c;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0, accm = 0, mmin = 0x7fffffff, mmax = 0;
        for (int k = 0; k < q; ++k) {
            lineptr[k] = acc;
            s_fp[k] = accm;
            fpk[k] = accm;
            acc += s_lines[k];
            accm += s_m[k];
            mmin = min(mmin, s_m[k]);
            mmax = max(mmax, s_m[k]);
        }
        lineptr[q] = acc;
        s_fp[q] = accm;
        fpk[q] = accm;
        meta[MT_NLINES] = acc;
        meta[MT_MMIN] = mmin;
        meta[MT_MMAX] = mmax;
        meta[MT_TOTAL] = accm;
        meta[MT_GENERAL] = s_partial;
        scal[SC_MBAR] = (double)accm / (double)q;
        int pacc = 0, nu = 0;
        for (int ky = 0; ky < ny; ++ky) {
            rfptr[ky] = pacc;
            pacc += s_rf[ky];
            rowused[ky] = (uint8_t)(s_rf[ky] > 0);
            if (s_rf[ky] > 0) usedrows[nu++] = ky;
        }
        rfptr[ny] = pacc;
        meta[MT_NUSED] = nu;
        if (fp_user[q] != (int64_t)accm || fp_user[0] != 0) atomicOr(status, (unsigned)ST_FRAMEPTR_MISMATCH);
    }
    __syncthreads();
    for (int k = tid; k < q; k += blockDim.x) {
        const int base = lineptr[k];
        if (fp_user[k] != (int64_t)s_fp[k]) atomicOr(status, (unsigned)ST_FRAMEPTR_MISMATCH);
        mks[k] = s_m[k];
        int i = 0, off = s_fp[k];
        for (int ky = 0; ky < ny; ++ky) {
            const int c = rowcnt[k * ny + ky];
            rowoff[k * ny + ky] = off;
            off += c;
            if (c > 0) {
                rowidx[k * ny + ky] = i;
                framerows[base + i] = ky;
                framek[base + i] = k;
                ++i;
            } else {
                rowidx[k * ny + ky] = -1;
            }
        }
    }
    for (int ky = tid; ky < ny; ky += blockDim.x) {
        int base = rfptr[ky], c = 0;
        for (int k = 0; k < q; ++k)
            if (rowcnt[k * ny + ky] > 0) rflist[base + c++] = k;
    }
}

__global__ void k_fill_idx(const int32_t *__restrict__ framerows, const int32_t *__restrict__ meta,
                           int nx, int32_t *idx) {
    const int g = blockIdx.x;
    if (g >= meta[MT_NLINES]) return;
    const int ky = framerows[g];
    for (int kx = threadIdx.x; kx < nx; kx += blockDim.x) idx[(size_t)g * nx + kx] = ky * nx + kx;
}

cudaError_t launch_compact(lrccs_ctx *c, const uint8_t *d_mask, const int64_t *d_fp_user) {
    const int rows = c->q * c->ny;
    prof_begin(c, KID_ROWCOUNT);
    k_rowcount<<<(rows * 32 + 255) / 256, 256, 0, c->stream>>>(d_mask, rows, c->nx, c->d_rowcnt);
    prof_end(c, KID_ROWCOUNT);
    prof_begin(c, KID_STRUCTURE);
    k_structure<<<1, 256, 0, c->stream>>>(c->d_rowcnt, d_fp_user, c->q, c->ny, c->nx, c->d_rowidx,
                                           c->d_framerows, c->d_framek, c->d_lineptr, c->d_rfptr, c->d_rflist,
                                           c->d_usedrows, c->d_rowused, c->d_mks, c->d_fpk, c->d_rowoff, c->d_meta,
                                           c->d_status, c->d_scal);
    prof_end(c, KID_STRUCTURE);
    return cudaGetLastError();
}

// Sample indices of masks that are unions of full lines (meta[MT_GENERAL] = 0).
cudaError_t launch_fill_lines(lrccs_ctx *c) {
    prof_begin(c, KID_FILL_IDX);
    k_fill_idx<<<c->q * c->ny, 128, 0, c->stream>>>(c->d_framerows, c->d_meta, c->nx, c->d_idx);
    prof_end(c, KID_FILL_IDX);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gamma
// gamma = trunc * sum |y|^2 / (number of measured entries)  (Alg. 2, init).
// |y|^2 is formed in FP64 without contraction so that the truncation decision
// |y|^2 <= gamma is taken on exactly the same squares as an FP64 reference.


__global__ void k_energy(const float2 *__restrict__ y, int64_t count, double trunc, double *part,
                         unsigned int *counter, double *scal) {
    __shared__ double s_red[32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += abs2_rn(y[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_red[w];
        part[blockIdx.x] = b;
    }
    if (last_block_arrive(counter) && threadIdx.x == 0) {
        double e = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) e += __ldcg(part + b);
        scal[SC_GAMMA] = trunc * e / (double)count;
    }
}

cudaError_t launch_energy(lrccs_ctx *c, const float2 *d_y) {
    const int64_t count = (int64_t)c->nc * c->total;
    const int blocks = 304;
    prof_begin(c, KID_ENERGY);
    k_energy<<<blocks, 256, 0, c->stream>>>(d_y, count, c->prm.trunc_factor, (double *)c->d_gpart,
                                            c->d_counters + CNT_ENERGY, c->d_scal);
    prof_end(c, KID_ENERGY);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Z and X0
// Z[:, k] = A_k^H y_k and X0[:, k] = A_k^H y_k,tnc / sqrt(m_k mbar), computed as
// a row pass (inverse DFT along kx of every sampled line, both the plain and
// the truncated data) and a column pass (inverse DFT along ky, coil combine
// with conj(d_j)).  The line layout of y makes every sampled row contiguous.

template <int P>
__global__ void __launch_bounds__(256) k_init_rows(const float2 *__restrict__ y, float2 *__restrict__ T0,
                                                    int64_t total_rows, const double *__restrict__ scal,
                                                    const float2 *__restrict__ g_tw, float scale) {
    // 4 rows x {plain, truncated} = 8 transforms per block; tile[x][2 row + ch]
    constexpr int N = 32 * P;
    constexpr int ROWS = 4, TPR = 2 * ROWS + 1;
    __shared__ float2 s_tw[N];
    __shared__ float2 tile[N * TPR];
    load_twiddles(s_tw, g_tw, N);
    const int64_t g0 = (int64_t)blockIdx.x * ROWS;
    const double gam = scal[SC_GAMMA];
    for (int e = threadIdx.x; e < ROWS * N; e += blockDim.x) {
        const int row = e / N, x = e - row * N;
        float2 a = make_float2(0.f, 0.f);
        if (g0 + row < total_rows) a = y[(g0 + row) * N + x];
        tile[x * TPR + 2 * row] = a;
        tile[x * TPR + 2 * row + 1] = abs2_rn(a) > gam ? make_float2(0.f, 0.f) : a;
    }
    __syncthreads();
    fft::tile_dft<N, true>(tile, TPR, 2 * ROWS, s_tw, scale);
    for (int e = threadIdx.x; e < ROWS * 2 * N; e += blockDim.x) {
        const int row = e / (2 * N), rem = e - row * 2 * N, x = rem >> 1, ch = rem & 1;
        if (g0 + row < total_rows) T0[(g0 + row) * N * 2 + rem] = tile[x * TPR + 2 * row + ch];
    }
}

#define TXI 8
template <int P>
__global__ void __launch_bounds__(256) k_init_cols(const float2 *__restrict__ T0, const float2 *__restrict__ smaps,
                                                    const int32_t *__restrict__ rowidx,
                                                    const int32_t *__restrict__ lineptr, const int32_t *__restrict__ mks,
                                                    const double *__restrict__ scal,
                                                    float2 *__restrict__ Z, float2 *__restrict__ X0, int nx, int q,
                                                    int nc, const float2 *__restrict__ g_tw, float scale) {
    constexpr int NY = 32 * P;
    constexpr int TP = 2 * TXI + 1;
    extern __shared__ float2 smem[];
    float2 *s_tw = smem;
    float2 *tile = s_tw + NY;
    float2 *s_S = tile + NY * TP;
    load_twiddles(s_tw, g_tw, NY);
    const int k = blockIdx.y, x0 = blockIdx.x * TXI;
    const int n = NY * nx;
    const int lp = lineptr[k];
    const int64_t mk = (int64_t)(lineptr[k + 1] - lp) * nx;
    const int64_t fbase = (int64_t)nc * lp * nx;
    // thread owns tile elements e = tid + 256 u: yy = e / (2 TXI), cc = e % (2 TXI)
    constexpr int ACC = (NY * 2 * TXI + 255) / 256;
    float2 acc[ACC];
    int goff[ACC];       // this thread's tile elements: offset in a coil's line block, or -1
#pragma unroll
    for (int u = 0; u < ACC; ++u) {
        acc[u] = make_float2(0.f, 0.f);
        const int e = threadIdx.x + 256 * u;
        goff[u] = -1;
        if (e < NY * 2 * TXI) {
            const int yy = e / (2 * TXI), cc = e % (2 * TXI);
            const int li = rowidx[k * NY + yy];
            if (li >= 0) goff[u] = (li * nx + x0) * 2 + cc;
        }
    }
    for (int j = 0; j < nc; ++j) {
        __syncthreads();
        const int64_t jb = (fbase + j * mk) * 2;
#pragma unroll
        for (int u = 0; u < ACC; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < NY * 2 * TXI) {
                const int yy = e / (2 * TXI), cc = e % (2 * TXI);
                tile[yy * TP + cc] = goff[u] >= 0 ? T0[jb + goff[u]] : make_float2(0.f, 0.f);
            }
        }
        for (int e = threadIdx.x; e < NY * TXI; e += blockDim.x)
            s_S[e] = smaps[(size_t)j * n + (size_t)(e / TXI) * nx + x0 + (e % TXI)];
        __syncthreads();
        fft::tile_dft<NY, true>(tile, TP, 2 * TXI, s_tw, scale);
#pragma unroll
        for (int u = 0; u < ACC; ++u) {
            const int e = threadIdx.x + 256 * u;
            if (e < NY * 2 * TXI) {
                const int yy = e / (2 * TXI), cc = e % (2 * TXI);
                cfmac(acc[u], s_S[yy * TXI + (cc >> 1)], tile[yy * TP + cc]);
            }
        }
    }
    const double mbar = scal[SC_MBAR];
    const int msamp = mks[k];   // samples per coil of frame k (m_k of Alg. 2's scale 1/sqrt(m_k mbar))
    const float xs = (msamp > 0) ? (float)(1.0 / sqrt((double)msamp * mbar)) : 0.f;
#pragma unroll
    for (int u = 0; u < ACC; ++u) {
        const int e = threadIdx.x + 256 * u;
        if (e < NY * 2 * TXI) {
            const int yy = e / (2 * TXI), cc = e % (2 * TXI);
            const size_t i = (size_t)yy * nx + x0 + (cc >> 1);
            if ((cc & 1) == 0) Z[i * q + k] = acc[u];
            else X0[i * q + k] = cscale(acc[u], xs);
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

cudaError_t launch_init_adjoint(lrccs_ctx *c, const float2 *d_y) {
    const int64_t total_rows = (int64_t)c->nc * c->n_lines;
    const float sx = (float)(1.0 / sqrt((double)c->nx));
    const float sy = (float)(1.0 / sqrt((double)c->ny));
    const unsigned rb = (unsigned)((total_rows + 3) / 4);
    if (c->general) return launch_init_general(c, d_y);   // frame rows hold scattered samples: one fused pass
    if (total_rows > 0) {
        DISPATCH_P(c->px, {
            prof_begin(c, KID_INIT_ROWS);
            k_init_rows<P_><<<rb, 256, 0, c->stream>>>(d_y, c->d_T, total_rows, c->d_scal, c->d_twx, sx);
            prof_end(c, KID_INIT_ROWS);
        });
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)c->ny * (1 + 2 * TXI + 1 + TXI) * sizeof(float2);
    dim3 grid(c->nx / TXI, c->q);
    DISPATCH_P(c->py, {
        prof_begin(c, KID_INIT_COLS);
        k_init_cols<P_><<<grid, 256, smem, c->stream>>>(c->d_T, c->d_smaps, c->d_rowidx, c->d_lineptr, c->d_mks,
                                                        c->d_scal, c->d_Z, c->d_X0, c->nx, c->q, c->nc,
                                                        c->d_twy, sy);
        prof_end(c, KID_INIT_COLS);
    });
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Gram of X0 and its eigensolver

#define GRAM_CHUNK 32
#define GRAM_THREADS 512
#define MAXPP 17   // pairs per thread: q(q+1)/2 <= 512 * 17 for q <= 128

template <int NS>   // pair slots per thread: q(q+1)/2 <= GRAM_THREADS NS
__global__ void __launch_bounds__(GRAM_THREADS) k_gram_x0(const float2 *__restrict__ X0, int n, int q,
                                                           float2 *part) {
    extern __shared__ float2 s_x[];  // GRAM_CHUNK * q, then the pair table
    short2 *s_pair = (short2 *)(s_x + GRAM_CHUNK * q);
    const int np = q * (q + 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        int a, b;
        pair_of(p, q, a, b);
        s_pair[p] = make_short2((short)a, (short)b);
    }
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    float2 acc[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) acc[u] = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += GRAM_CHUNK) {
        const int cn = min(GRAM_CHUNK, i1 - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cn * q; e += blockDim.x) s_x[e] = X0[(size_t)c0 * q + e];
        __syncthreads();
        for (int ii = 0; ii < cn; ++ii) {   // all of this thread's pairs per pixel (independent chains)
            const float2 *xr = s_x + ii * q;
#pragma unroll
            for (int u = 0; u < NS; ++u) {
                const int p = threadIdx.x + GRAM_THREADS * u;
                if (p < np) {
                    const short2 ab = s_pair[p];
                    cfmac(acc[u], xr[ab.x], xr[ab.y]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int p = threadIdx.x + GRAM_THREADS * u;
        if (p < np) part[(size_t)blockIdx.x * np + p] = acc[u];
    }
}

// Sum the nblk partial rows of k_gram_x0 into the FP64 Hermitian Gram: thread
// (pair p, slice s of 4) adds blocks s, s + 4, ... in compensated FP32 with 8
// loads in flight; the 4 slices are then added in order.
__global__ void __launch_bounds__(256) k_gram_sum(const float2 *__restrict__ part, int nblk, int q,
                                                  double *__restrict__ gram) {
    __shared__ float4 s_acc[256];
    const int np = q * (q + 1) / 2;
    const int pl = threadIdx.x & 63, sl = threadIdx.x >> 6;
    const int p = blockIdx.x * 64 + pl;
    fsum2 re = {0.f, 0.f}, im = {0.f, 0.f};
    if (p < np) {
        int b = sl;
        for (; b + 28 < nblk; b += 32) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (size_t)(b + 4 * u) * np + p);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                fsum_add(re, v[u].x);
                fsum_add(im, v[u].y);
            }
        }
        for (; b < nblk; b += 4) {
            const float2 v = __ldcg(part + (size_t)b * np + p);
            fsum_add(re, v.x);
            fsum_add(im, v.y);
        }
    }
    s_acc[threadIdx.x] = make_float4(re.hi, re.lo, im.hi, im.lo);
    __syncthreads();
    if (sl == 0 && p < np) {
        fsum2 R = {s_acc[pl].x, s_acc[pl].y}, I = {s_acc[pl].z, s_acc[pl].w};
        for (int k = 1; k < 4; ++k) {
            const float4 w = s_acc[k * 64 + pl];
            R = fsum_pair(R, fsum2{w.x, w.y});
            I = fsum_pair(I, fsum2{w.z, w.w});
        }
        int a, bb;
        pair_of(p, q, a, bb);
        const double sr = (double)R.hi + (double)R.lo, si = (double)I.hi + (double)I.lo;
        gram[2 * (a * q + bb)] = sr;
        gram[2 * (a * q + bb) + 1] = si;
        gram[2 * (bb * q + a)] = sr;
        gram[2 * (bb * q + a) + 1] = -si;
    }
}

// Eigendecomposition of the q x q Gram A = X0^H X0 (Alg. 2: sigma_j^2 and the
// right singular vectors of X0) in two passes, each a parallel cyclic Jacobi
// in FP32 in one block:
//   pass 0 : Jacobi on A (rounded to FP32) -> V0.  Its rotations leave errors
//            of about eps ||A|| in every entry, so the eigenvectors of small
//            eigenvalues are off by about eps lambda_1 / gap;
//   refine : B = V0^H A V0 formed in FP64 (k_refine_av, k_refine_vhb), whose
//            off-diagonal entries are those small errors, held in FP32 with
//            full relative precision; a second Jacobi (relative threshold
//            only) on B -> Q, and V = V0 Q.  The second pass's rounding is
//            relative to the entries it rotates, so every eigenpair comes out
//            accurate relative to its own eigenvalue and gap (mixed-precision
//            Jacobi refinement).
// The refine pass also sorts: sigma_j = sqrt(lambda_j) descending, and the
// rank rule of Alg. 2 when rank_in == 0: the smallest r whose leading sigma^2
// reach b% of the energy of the first floor(min(n, q, C min m_k)/10) (at least 1).
__global__ void k_eig(const double *__restrict__ gram, int q, int n, int nc, int rank_in, int rmax,
                      double energy_pct, float2 *V, float2 *Q, int32_t *order, double *sigma, int32_t *meta,
                      unsigned int *status, int v_in_smem, int refine) {
    // A (and the rotation matrix when it fits) in shared memory with an odd row
    // pitch, so that the column updates of the rotations hit distinct banks
    extern __shared__ float2 sA[];
    __shared__ float s_c[64], s_s[64];
    __shared__ float2 s_e[64];
    __shared__ int s_cnt;
    __shared__ double s_fro[32];
    __shared__ double s_scale;
    __shared__ float s_lam[128];
    const int ld = q | 1;
    float2 *Vw = v_in_smem ? sA + q * ld : (refine ? Q : V);
    const int ldv = v_in_smem ? ld : q;
    if (threadIdx.x == 0) {   // the refine pass works on B / max diag(B)
        double mx = 0.0;
        if (refine)
            for (int i = 0; i < q; ++i) mx = fmax(mx, gram[2 * (i * q + i)]);
        s_scale = mx > 0.0 ? mx : 1.0;
    }
    __syncthreads();
    const double isc = refine ? 1.0 / s_scale : 1.0;
    double fro = 0.0;
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int a = e / q, b = e - a * q;
        sA[a * ld + b] = make_float2((float)(gram[2 * e] * isc), (float)(gram[2 * e + 1] * isc));
        Vw[a * ldv + b] = make_float2(a == b ? 1.f : 0.f, 0.f);
        fro += gram[2 * e] * gram[2 * e] + gram[2 * e + 1] * gram[2 * e + 1];
    }
    fro = warp_sum_d(fro);
    if ((threadIdx.x & 31) == 0) s_fro[threadIdx.x >> 5] = fro;
    __syncthreads();
    fro = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fro += s_fro[w];
    if (!refine) {
        // a rotation is skipped once |a_pq| <= 1e-5 sqrt(a_pp a_qq) or <= 1e-6
        // ||A||_F, at most 5 sweeps: this pass only has to leave B = V0^H A V0
        // diagonally dominant; the refine pass converges quadratically from there
        block_jacobi(sA, q, ld, Vw, ldv, s_c, s_s, s_e, &s_cnt, 5, (float)(1e-6 * sqrt(fro)), 1e-5f);
        if (v_in_smem)
            for (int e = threadIdx.x; e < q * q; e += blockDim.x) V[e] = Vw[(e / q) * ldv + e % q];
        return;
    }
    // the wanted eigenpairs: the top rank_in (fixed rank) or the rank rule's
    // cap; rotations between two indices whose diagonal entries are both
    // below a quarter of the r_w-th largest entry cannot change them
    __shared__ float s_tail;
    {
        int capn = min(n, q);
        const long long cm = (long long)nc * meta[MT_MMIN];
        if (cm < capn) capn = (int)cm;
        const int cap = max(1, capn / 10);
        const int rw = min(q, max(rank_in, cap));
        for (int i = threadIdx.x; i < q; i += blockDim.x) {
            const float di = sA[i * ld + i].x;
            int above = 0;
            for (int j = 0; j < q; ++j) {
                const float dj = sA[j * ld + j].x;
                above += (dj > di || (dj == di && j < i)) ? 1 : 0;
            }
            if (above == rw - 1) s_tail = 0.25f * di;
        }
        __syncthreads();
    }
    block_jacobi(sA, q, ld, Vw, ldv, s_c, s_s, s_e, &s_cnt, 6, 0.f, 1e-6f, s_tail);
    // eigenvalues (diagonal of the rotated B, scaled back), then V <- V0 Q,
    // formed in the shared A region (A is no longer needed)
    for (int i = threadIdx.x; i < q; i += blockDim.x) s_lam[i] = sA[i * ld + i].x;
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int a = e / q, b = e - a * q;
        float2 acc = make_float2(0.f, 0.f);
        for (int m = 0; m < q; ++m) cfma(acc, V[a * q + m], Vw[m * ldv + b]);
        sA[a * ld + b] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) V[e] = sA[(e / q) * ld + e % q];
    // eigenvalue order, descending (ties by index): thread i finds its rank
    for (int i = threadIdx.x; i < q; i += blockDim.x) {
        const float li = s_lam[i];
        int rank = 0;
        for (int j = 0; j < q; ++j) {
            const float lj = s_lam[j];
            rank += (lj > li || (lj == li && j < i)) ? 1 : 0;
        }
        order[rank] = i;
        sigma[rank] = sqrt(li > 0.f ? (double)li * s_scale : 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = rank_in;
        if (r <= 0) {
            long long capn = min(n, q);
            long long cm = (long long)nc * meta[MT_MMIN];
            if (cm < capn) capn = cm;
            int cap = (int)(capn / 10);
            if (cap < 1) cap = 1;
            double tot = 0.0, acc = 0.0;
            for (int j = 0; j < cap; ++j) tot += sigma[j] * sigma[j];
            r = cap;
            for (int j = 0; j < cap; ++j) {
                acc += sigma[j] * sigma[j];
                if (acc >= energy_pct / 100.0 * tot) { r = j + 1; break; }
            }
        }
        meta[MT_RANK] = r;
        if (r > rmax || r > q) atomicOr(status, (unsigned)ST_ZERO_SIGMA);
        else if (!(sigma[r - 1] > 0.0)) atomicOr(status, (unsigned)ST_ZERO_SIGMA);
    }
}

// T = A V0 in FP64 (A: the FP64 Gram, (re, im) pairs; V0: FP32 eigenvectors
// of pass 0): block a forms row a of T.
__global__ void k_refine_av(const double *__restrict__ gram, const float2 *__restrict__ V, int q, double *T) {
    const int a = blockIdx.x;
    for (int b = threadIdx.x; b < q; b += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < q; ++j) {
            const double ar = gram[2 * (a * q + j)], ai = gram[2 * (a * q + j) + 1];
            const float2 v = V[j * q + b];
            re += ar * v.x - ai * v.y;
            im += ar * v.y + ai * v.x;
        }
        T[2 * (a * q + b)] = re;
        T[2 * (a * q + b) + 1] = im;
    }
}

// B = V0^H T in FP64, made exactly Hermitian (the mean of B and B^H): block a
// forms row a; entries (a, b) and (b, a) are summed in the same order.
__global__ void k_refine_vhb(const float2 *__restrict__ V, const double *__restrict__ T, int q, double *Bm) {
    const int a = blockIdx.x;
    for (int b = threadIdx.x; b < q; b += blockDim.x) {
        double re = 0.0, im = 0.0, re2 = 0.0, im2 = 0.0;
        for (int i = 0; i < q; ++i) {
            const float2 va = V[i * q + a], vb = V[i * q + b];
            const double tr = T[2 * (i * q + b)], ti = T[2 * (i * q + b) + 1];   // T[i][b]
            const double ur = T[2 * (i * q + a)], ui = T[2 * (i * q + a) + 1];   // T[i][a]
            re += va.x * tr + va.y * ti;    // conj(V[i][a]) T[i][b] = B[a][b]
            im += va.x * ti - va.y * tr;
            re2 += vb.x * ur + vb.y * ui;   // conj(V[i][b]) T[i][a] = B[b][a]
            im2 += vb.x * ui - vb.y * ur;
        }
        Bm[2 * (a * q + b)] = 0.5 * (re + re2);
        Bm[2 * (a * q + b) + 1] = 0.5 * (im - im2);
    }
}

cudaError_t launch_gram_x0(lrccs_ctx *c) {
    const int q = c->q;
    const int np = q * (q + 1) / 2;
    int blocks = (c->n + 127) / 128;
    if (blocks > 152) blocks = 152;
    if ((size_t)blocks * np > c->gpart_cap) blocks = (int)(c->gpart_cap / np);
    const size_t smem = (size_t)GRAM_CHUNK * q * sizeof(float2) + (size_t)np * sizeof(short2);
    double *gram = c->d_gram;
    prof_begin(c, KID_GRAM_X0);
    const int ns = (np + GRAM_THREADS - 1) / GRAM_THREADS;
    if (ns <= 1) k_gram_x0<1><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else if (ns <= 2) k_gram_x0<2><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else if (ns <= 3) k_gram_x0<3><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else if (ns <= 5) k_gram_x0<5><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else if (ns <= 8) k_gram_x0<8><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else if (ns <= 12) k_gram_x0<12><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    else k_gram_x0<MAXPP><<<blocks, GRAM_THREADS, smem, c->stream>>>(c->d_X0, c->n, q, c->d_gpart);
    k_gram_sum<<<(np + 63) / 64, 256, 0, c->stream>>>(c->d_gpart, blocks, q, gram);
    prof_end(c, KID_GRAM_X0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ld = q | 1;
    const int v_in_smem = (size_t)2 * q * ld * sizeof(float2) + 4096 <= (size_t)c->dev_smem_optin;
    const size_t smem2 = (size_t)(v_in_smem ? 2 : 1) * q * ld * sizeof(float2);
    double *T = c->d_gram + 2 * (size_t)q * q, *Bm = T + 2 * (size_t)q * q;
    prof_begin(c, KID_EIG);
    k_eig<<<1, 1024, smem2, c->stream>>>(gram, q, c->n, c->nc, c->dims.rank, c->rmax, c->prm.energy_pct, c->d_V,
                                        c->d_Q, c->d_meta + MT_COUNT, c->d_sigma, c->d_meta, c->d_status, v_in_smem,
                                        0);
    prof_end(c, KID_EIG);
    prof_begin(c, KID_EIG);
    k_refine_av<<<q, 128, 0, c->stream>>>(gram, c->d_V, q, T);
    prof_end(c, KID_EIG);
    prof_begin(c, KID_EIG);
    k_refine_vhb<<<q, 128, 0, c->stream>>>(c->d_V, T, q, Bm);
    prof_end(c, KID_EIG);
    prof_begin(c, KID_EIG);
    k_eig<<<1, 1024, smem2, c->stream>>>(Bm, q, c->n, c->nc, c->dims.rank, c->rmax, c->prm.energy_pct, c->d_V,
                                        c->d_Q, c->d_meta + MT_COUNT, c->d_sigma, c->d_meta, c->d_status, v_in_smem,
                                        1);
    prof_end(c, KID_EIG);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- U_0
// U_0 = X0 V_r Sigma_r^{-1}: the top-r left singular vectors of X0 (Alg. 2),
// written to the U+ buffer and then orthonormalised by CholeskyQR2.

__global__ void k_u0(const float2 *__restrict__ X0, const float2 *__restrict__ V, const int32_t *__restrict__ order,
                     const double *__restrict__ sigma, int n, int q, int r, float2 *Up) {
    extern __shared__ float2 s_v[];  // q * r, scaled by 1/sigma
    for (int e = threadIdx.x; e < q * r; e += blockDim.x) {
        const int k = e / r, l = e % r;
        const float is = (float)(1.0 / sigma[l]);
        s_v[e] = cscale(V[k * q + order[l]], is);
    }
    __syncthreads();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * r; e += gridDim.x * blockDim.x) {
        const int i = e / r, l = e % r;
        float2 acc = make_float2(0.f, 0.f);
        const float2 *xr = X0 + (size_t)i * q;
        for (int k = 0; k < q; ++k) cfma(acc, xr[k], s_v[k * r + l]);
        Up[e] = acc;
    }
}

cudaError_t launch_u0(lrccs_ctx *c) {
    const size_t smem = (size_t)c->q * c->r * sizeof(float2);
    prof_begin(c, KID_U0);
    k_u0<<<304, 256, smem, c->stream>>>(c->d_X0, c->d_V, c->d_meta + MT_COUNT, c->d_sigma, c->n, c->q, c->r,
                                        c->d_Up);
    prof_end(c, KID_U0);
    return cudaGetLastError();
}

// Allow every kernel of this file the device's opt-in shared memory per block
// (the launch still requests only what it needs).
#define SET_SMEM(fn) do { cudaError_t e_ = allow_smem(fn, max_smem); if (e_ != cudaSuccess) return e_; } while (0)
cudaError_t configure_kernels_init(int max_smem) {
    SET_SMEM(k_init_cols<1>); SET_SMEM(k_init_cols<2>); SET_SMEM(k_init_cols<3>); SET_SMEM(k_init_cols<4>);
    SET_SMEM(k_init_cols<5>); SET_SMEM(k_init_cols<6>); SET_SMEM(k_init_cols<7>); SET_SMEM(k_init_cols<8>);
    SET_SMEM(k_gram_x0<1>); SET_SMEM(k_gram_x0<2>); SET_SMEM(k_gram_x0<3>); SET_SMEM(k_gram_x0<5>);
    SET_SMEM(k_gram_x0<8>); SET_SMEM(k_gram_x0<12>); SET_SMEM(k_gram_x0<MAXPP>);
    SET_SMEM(k_eig);
    SET_SMEM(k_u0);
    return cudaGetLastError();
}
