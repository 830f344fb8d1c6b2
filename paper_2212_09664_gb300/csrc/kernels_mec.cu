// kernels_mec.cu -- model-error correction (Alg. 3) and the per-frame normal
// operator it needs, on sm_103a.
//
// After Alg. 2, the residual measurements ytt_k = y~_k - A_k x_k (x_k = U b_k)
// still hold what the low-rank model misses.  Alg. 3 estimates it as
//   MEC-1: e_k from a few CGLS iterations on min_e ||ytt_k - A_k e||^2, per frame;
//   MEC-2: ISTA on min_E sum_k ||ytt_k - A_k e_k||^2 + omega ||F_t E||_1 with F_t
//          the DFT along the frames (a temporally sparse residual).
// Both only need the frames' normal operators N_k = A_k^H A_k and
// s_k = A_k^H ytt_k = Z[:, k] - N_k x_k (Z = [A_k^H y~_k] from the init).
//
// Frames are processed in chunks of w = rank_max columns, vectors laid out as
// V[c][i][l] (frame k = c w + l, pixel i), so that the iteration's column
// transforms apply N to a whole chunk at once:
//   N_k v = sum_j conj(d_j) o F^H [M_k o F(d_j o v)],
// with the per-frame sampling M_k applied between the forward and inverse
// transforms (k_mask_rows for line masks, k_mask_points for general ones).
// Reductions per frame (dot products, norms) are FP64 in a fixed order.
#include <math.h>

#include "common.cuh"
#include "internal.h"

#define MEC_G 152   // pixel blocks of the reduction kernels (one wave on 152 SMs)

// ---------------------------------------------------------------- per-frame sampling between the transforms

// Line masks: T_j[ky][x][l] of the used rows is kept only if frame k0 + l
// samples row ky (frames >= q sample nothing).
__global__ void k_mask_rows(float2 *__restrict__ T, const int32_t *__restrict__ usedrows,
                            const int32_t *__restrict__ rowidx, int ny, int nx, int nc, int w, int k0, int q) {
    const int ky = usedrows[blockIdx.x], j = blockIdx.y;
    float2 *row = T + ((size_t)j * ny + ky) * nx * w;
    for (int e = threadIdx.x; e < nx * w; e += blockDim.x) {
        const int l = e % w, k = k0 + l;
        if (k >= q || rowidx[k * ny + ky] < 0) row[e] = make_float2(0.f, 0.f);
    }
}

// General masks: FU_j[u][l] is kept only if frame k0 + l samples union point u.
__global__ void k_mask_points(float2 *__restrict__ FU, const uint8_t *__restrict__ maskc,
                              const int32_t *__restrict__ uidx, int n, int nu, int nc, int w, int k0, int q) {
    const size_t total = (size_t)nc * nu * w;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % w);
        const int u = (int)((e / w) % nu);
        const int k = k0 + l;
        if (k >= q || !maskc[(size_t)k * n + uidx[u]]) FU[e] = make_float2(0.f, 0.f);
    }
}

// dst (n x w) <- [N_{k0+l} src[:, l]]_l for one chunk of frames.
cudaError_t launch_frame_normal_op(lrccs_ctx *c, const float2 *src, float2 *dst, int w, int k0) {
    cudaError_t e = launch_fwd_cols_on(c, src, w);
    if (e != cudaSuccess) return e;
    if (c->general) {
        e = launch_fwd_rows_r(c, w);
        if (e != cudaSuccess) return e;
        prof_begin(c, KID_MEC_MASK);
        k_mask_points<<<4 * 152, 256, 0, c->stream>>>(c->d_FU, c->d_maskc, c->d_uidx, c->n, c->n_u, c->nc, w, k0,
                                                       c->q);
        prof_end(c, KID_MEC_MASK);
        e = launch_adj_rows_r(c, w);
        if (e != cudaSuccess) return e;
    } else {
        prof_begin(c, KID_MEC_MASK);
        k_mask_rows<<<dim3(c->n_used, c->nc), 256, 0, c->stream>>>(c->d_T, c->d_usedrows, c->d_rowidx, c->ny, c->nx,
                                                                    c->nc, w, k0, c->q);
        prof_end(c, KID_MEC_MASK);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_adj_cols_to(c, dst, w);
}

// ---------------------------------------------------------------- elementwise and reductions

// X[c][i][l] = U_{t-1}[i, :] b_k (k = c w + l < q, else 0); with zbar != NULL
// (and Uprev == NULL) X[c][i][l] = zbar[i] for every frame instead.
__global__ void k_mec_x(const float2 *__restrict__ Uprev, const float2 *__restrict__ B, const float2 *__restrict__ zbar,
                        int n, int q, int r, int w, int nch, float2 *__restrict__ X) {
    const size_t total = (size_t)nch * n * w;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % w);
        const size_t ci = e / w;
        const int i = (int)(ci % n), cc = (int)(ci / n);
        const int k = cc * w + l;
        float2 v = make_float2(0.f, 0.f);
        if (k < q) {
            if (Uprev) {
                for (int a = 0; a < r; ++a) cfma(v, Uprev[(size_t)i * r + a], B[(size_t)k * r + a]);
            } else {
                v = zbar[i];
            }
        }
        X[e] = v;
    }
}

// Z[i][k] -= V[c][i][l] (the mean's normal-operator image, online tracking).
__global__ void k_mec_subz(float2 *__restrict__ Z, const float2 *__restrict__ V, int n, int q, int w) {
    const size_t total = (size_t)n * q;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / q), k = (int)(e % q);
        const float2 v = V[((size_t)(k / w) * n + i) * w + (k % w)];
        Z[e] = csub(Z[e], v);
    }
}

// Block (pixel range b, chunk cc); thread (column l, slice): per-frame FP64
// partial sums of the value returned by f(index), written to part[b][cc w + l].
template <class F>
__device__ void mec_block_partial(int n, int w, double *part, F f) {
    __shared__ double s_red[256];
    const int b = blockIdx.x, cc = blockIdx.y, G = gridDim.x, NW = gridDim.y * w;
    const int per = (n + G - 1) / G;
    const int i0 = min(n, b * per), i1 = min(n, i0 + per);
    const int S = blockDim.x / w, l = threadIdx.x % w, sl = threadIdx.x / w;
    double acc = 0.0;
    if (sl < S)
        for (int i = i0 + sl; i < i1; i += S) acc += f(((size_t)cc * n + i) * w + l);
    s_red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < w) {
        double s = 0.0;
        for (int v = 0; v < S; ++v) s += s_red[v * w + threadIdx.x];
        part[(size_t)b * NW + cc * w + threadIdx.x] = s;
    }
}

// S = Z - V, P = S, E = 0 and the partials of gamma_k = ||S_k||^2.
__global__ void __launch_bounds__(256) k_mec_start(const float2 *__restrict__ Z, const float2 *__restrict__ V, int n,
                                                   int q, int w, float2 *__restrict__ S, float2 *__restrict__ P,
                                                   float2 *__restrict__ E, double *part) {
    mec_block_partial(n, w, part, [&](size_t e) {
        const int l = (int)(e % w), i = (int)((e / w) % n), k = (int)(e / ((size_t)n * w)) * w + l;
        float2 s = make_float2(0.f, 0.f);
        if (k < q) s = csub(Z[(size_t)i * q + k], V[e]);
        S[e] = s;
        P[e] = s;
        E[e] = make_float2(0.f, 0.f);
        return (double)s.x * s.x + (double)s.y * s.y;
    });
}

// partials of Re<p_k, w_k> (= ||A_k p_k||^2)
__global__ void __launch_bounds__(256) k_mec_dot(const float2 *__restrict__ P, const float2 *__restrict__ W, int n,
                                                 int w, double *part) {
    mec_block_partial(n, w, part, [&](size_t e) {
        const float2 a = P[e], b = W[e];
        return (double)a.x * b.x + (double)a.y * b.y;
    });
}

// e += alpha p, s -= alpha w, and the partials of the new ||s_k||^2
__global__ void __launch_bounds__(256) k_mec_update(const float2 *__restrict__ P, const float2 *__restrict__ W,
                                                    float2 *__restrict__ E, float2 *__restrict__ S,
                                                    const double *__restrict__ alpha, int n, int w, double *part) {
    mec_block_partial(n, w, part, [&](size_t e) {
        const int k = (int)(e / ((size_t)n * w)) * w + (int)(e % w);
        const float a = (float)alpha[k];
        const float2 p = P[e], ww = W[e];
        float2 ee = E[e], ss = S[e];
        ee.x = fmaf(a, p.x, ee.x);
        ee.y = fmaf(a, p.y, ee.y);
        ss.x = fmaf(-a, ww.x, ss.x);
        ss.y = fmaf(-a, ww.y, ss.y);
        E[e] = ee;
        S[e] = ss;
        return (double)ss.x * ss.x + (double)ss.y * ss.y;
    });
}

// p = s + beta p
__global__ void k_mec_dir(const float2 *__restrict__ S, float2 *__restrict__ P, const double *__restrict__ beta, int n,
                          int w, int nch) {
    const size_t total = (size_t)nch * n * w;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / ((size_t)n * w)) * w + (int)(e % w);
        const float bb = (float)beta[k];
        const float2 s = S[e], p = P[e];
        P[e] = make_float2(fmaf(bb, p.x, s.x), fmaf(bb, p.y, s.y));
    }
}

// Per frame k < q: total = sum over the G pixel blocks of part[b][k] (in b
// order), then   mode 0: gamma = total;   mode 1: alpha = gamma / total (0 if
// the frame's direction has no energy);   mode 2: beta = total / gamma, gamma = total.
__global__ void k_mec_finish(const double *__restrict__ part, int G, int NW, int q, int mode, double *gamma,
                             double *alpha, double *beta) {
    for (int k = threadIdx.x; k < q; k += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < G; ++b) t += part[(size_t)b * NW + k];
        if (mode == 0) {
            gamma[k] = t;
        } else if (mode == 1) {
            alpha[k] = (t > 0.0 && gamma[k] > 0.0) ? gamma[k] / t : 0.0;
        } else {
            beta[k] = gamma[k] > 0.0 ? t / gamma[k] : 0.0;
            gamma[k] = t;
        }
    }
}

// Caller layouts (frame k contiguous, X[k n + i]): E_out = e_k and
// X_out = zbar + U_{t-1} b_k + e_k (zbar may be NULL).
__global__ void k_mec_out(const float2 *__restrict__ E, const float2 *__restrict__ Uprev, const float2 *__restrict__ B,
                          const float2 *__restrict__ zbar, int n, int q, int r, int w, float2 *__restrict__ Eout,
                          float2 *__restrict__ Xout) {
    const size_t total = (size_t)n * q;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n), i = (int)(e % n);
        const float2 ev = E[((size_t)(k / w) * n + i) * w + (k % w)];
        if (Eout) Eout[e] = ev;
        if (Xout) {
            float2 x = zbar ? zbar[i] : make_float2(0.f, 0.f);
            for (int a = 0; a < r; ++a) cfma(x, Uprev[(size_t)i * r + a], B[(size_t)k * r + a]);
            Xout[e] = cadd(x, ev);
        }
    }
}

// ---------------------------------------------------------------- MEC-2: DFT along the frames

#define TD_PIX 8   // pixels per block of the temporal transforms

// M[:, i] = F_t (E + S0 - V)[i, :] (unitary DFT over the q frames, tw[t] =
// exp(-2 pi i t / q)) for TD_PIX pixels per block, and the block's max |M|,
// sum |M - Mprev|^2 and sum |Mprev|^2 (when have_prev) into part[blk][3].
__global__ void __launch_bounds__(256) k_tdft_fwd(const float2 *__restrict__ E, const float2 *__restrict__ S0,
                                                  const float2 *__restrict__ V, const float2 *__restrict__ Mprev,
                                                  const float2 *__restrict__ tw, int n, int q, int w, int have_v,
                                                  int have_prev, float2 *__restrict__ M, double *part) {
    extern __shared__ float2 s_g[];           // TD_PIX * q, then tw (q)
    float2 *s_tw = s_g + TD_PIX * q;
    __shared__ double s_r[3][256];
    const int i0 = blockIdx.x * TD_PIX;
    const float sc = rsqrtf((float)q);
    for (int t = threadIdx.x; t < q; t += blockDim.x) s_tw[t] = tw[t];
    for (int e = threadIdx.x; e < TD_PIX * q; e += blockDim.x) {
        const int p = e / q, k = e - p * q, i = i0 + p;
        float2 g = make_float2(0.f, 0.f);
        if (i < n) {
            const size_t o = ((size_t)(k / w) * n + i) * w + (k % w);
            g = cadd(E[o], S0[o]);
            if (have_v) g = csub(g, V[o]);
        }
        s_g[e] = g;
    }
    __syncthreads();
    double mx = 0.0, dd = 0.0, pp = 0.0;
    for (int e = threadIdx.x; e < TD_PIX * q; e += blockDim.x) {
        const int p = e / q, f = e - p * q, i = i0 + p;
        if (i >= n) continue;
        float2 acc = make_float2(0.f, 0.f);
        int t = 0;
        for (int k = 0; k < q; ++k) {
            cfma(acc, s_g[p * q + k], s_tw[t]);
            t += f;
            if (t >= q) t -= q;
        }
        acc = cscale(acc, sc);
        const size_t o = ((size_t)(f / w) * n + i) * w + (f % w);
        M[o] = acc;
        mx = fmax(mx, sqrt((double)acc.x * acc.x + (double)acc.y * acc.y));
        if (have_prev) {
            const float2 m0 = Mprev[o];
            const double dx = (double)acc.x - m0.x, dy = (double)acc.y - m0.y;
            dd += dx * dx + dy * dy;
            pp += (double)m0.x * m0.x + (double)m0.y * m0.y;
        }
    }
    s_r[0][threadIdx.x] = mx;
    s_r[1][threadIdx.x] = dd;
    s_r[2][threadIdx.x] = pp;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            a = fmax(a, s_r[0][t]);
            b += s_r[1][t];
            cc += s_r[2][t];
        }
        part[(size_t)blockIdx.x * 3 + 0] = a;
        part[(size_t)blockIdx.x * 3 + 1] = b;
        part[(size_t)blockIdx.x * 3 + 2] = cc;
    }
}

// out[0] = max, out[1], out[2] = sums of the nb block partials (fixed order).
__global__ void k_tdft_finish(const double *__restrict__ part, int nb, double *out) {
    __shared__ double s_r[3][256];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        a = fmax(a, part[(size_t)t * 3]);
        b += part[(size_t)t * 3 + 1];
        c += part[(size_t)t * 3 + 2];
    }
    s_r[0][threadIdx.x] = a;
    s_r[1][threadIdx.x] = b;
    s_r[2][threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {   // thread 0's own partials are in a, b, c already
        for (int t = 1; t < (int)blockDim.x; ++t) {
            a = fmax(a, s_r[0][t]);
            b += s_r[1][t];
            c += s_r[2][t];
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

// E[i, :] = F_t^{-1} SThr_omega(M[:, i]): the complex soft threshold
// m (|m| - omega) / |m| for |m| > omega, else 0, then the inverse unitary DFT.
__global__ void __launch_bounds__(256) k_tdft_inv(const float2 *__restrict__ M, const float2 *__restrict__ tw, int n,
                                                  int q, int w, float omega, float2 *__restrict__ E) {
    extern __shared__ float2 s_g[];
    float2 *s_tw = s_g + TD_PIX * q;
    const int i0 = blockIdx.x * TD_PIX;
    const float sc = rsqrtf((float)q);
    for (int t = threadIdx.x; t < q; t += blockDim.x) s_tw[t] = tw[t];
    for (int e = threadIdx.x; e < TD_PIX * q; e += blockDim.x) {
        const int p = e / q, f = e - p * q, i = i0 + p;
        float2 m = make_float2(0.f, 0.f);
        if (i < n) {
            m = M[((size_t)(f / w) * n + i) * w + (f % w)];
            const float a = sqrtf(m.x * m.x + m.y * m.y);
            m = a > omega ? cscale(m, (a - omega) / a) : make_float2(0.f, 0.f);
        }
        s_g[e] = m;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TD_PIX * q; e += blockDim.x) {
        const int p = e / q, k = e - p * q, i = i0 + p;
        if (i >= n) continue;
        float2 acc = make_float2(0.f, 0.f);
        int t = 0;
        for (int f = 0; f < q; ++f) {
            cfma(acc, s_g[p * q + f], cconj(s_tw[t]));
            t += k;
            if (t >= q) t -= q;
        }
        E[((size_t)(k / w) * n + i) * w + (k % w)] = cscale(acc, sc);
    }
}

// ---------------------------------------------------------------- launchers

static int mec_blocks(int n) { return n < MEC_G * 64 ? (n + 63) / 64 : MEC_G; }

cudaError_t launch_mec_x(lrccs_ctx *c, const float2 *Uprev, const float2 *zbar, float2 *X) {
    prof_begin(c, KID_MEC_ELEM);
    k_mec_x<<<4 * 152, 256, 0, c->stream>>>(Uprev, c->d_B, zbar, c->n, c->q, c->r, c->mec_w, c->mec_nch, X);
    prof_end(c, KID_MEC_ELEM);
    return cudaGetLastError();
}

cudaError_t launch_mec_subz(lrccs_ctx *c, const float2 *V) {
    prof_begin(c, KID_MEC_ELEM);
    k_mec_subz<<<4 * 152, 256, 0, c->stream>>>(c->d_Z, V, c->n, c->q, c->mec_w);
    prof_end(c, KID_MEC_ELEM);
    return cudaGetLastError();
}

// kind: 0 start (S = Z - V, P = S, E = 0, gamma), 1 alpha (from P, W), 2
// update (E, S, then beta and gamma), 3 direction (P = S + beta P).
cudaError_t launch_mec_cg(lrccs_ctx *c, int kind, const float2 *V) {
    const int n = c->n, w = c->mec_w, nch = c->mec_nch, G = mec_blocks(n), NW = nch * w;
    double *gamma = c->d_mscal, *alpha = gamma + c->q, *beta = alpha + c->q, *part = beta + c->q;
    float2 *E = c->d_mec, *S = E + (size_t)nch * n * w, *P = S + (size_t)nch * n * w, *W = P + (size_t)nch * n * w;
    dim3 grid(G, nch);
    prof_begin(c, KID_MEC_ELEM);
    if (kind == 0) {
        k_mec_start<<<grid, 256, 0, c->stream>>>(c->d_Z, V, n, c->q, w, S, P, E, part);
        k_mec_finish<<<1, 128, 0, c->stream>>>(part, G, NW, c->q, 0, gamma, alpha, beta);
    } else if (kind == 1) {
        k_mec_dot<<<grid, 256, 0, c->stream>>>(P, W, n, w, part);
        k_mec_finish<<<1, 128, 0, c->stream>>>(part, G, NW, c->q, 1, gamma, alpha, beta);
    } else if (kind == 2) {
        k_mec_update<<<grid, 256, 0, c->stream>>>(P, W, E, S, alpha, n, w, part);
        k_mec_finish<<<1, 128, 0, c->stream>>>(part, G, NW, c->q, 2, gamma, alpha, beta);
    } else {
        k_mec_dir<<<4 * 152, 256, 0, c->stream>>>(S, P, beta, n, w, nch);
    }
    prof_end(c, KID_MEC_ELEM);
    return cudaGetLastError();
}

cudaError_t launch_mec_out(lrccs_ctx *c, const float2 *E, const float2 *zbar, float2 *Eout, float2 *Xout) {
    prof_begin(c, KID_MEC_ELEM);
    k_mec_out<<<4 * 152, 256, 0, c->stream>>>(E, c->d_Uprev, c->d_B, zbar, c->n, c->q, c->r, c->mec_w, Eout, Xout);
    prof_end(c, KID_MEC_ELEM);
    return cudaGetLastError();
}

cudaError_t launch_tdft_fwd(lrccs_ctx *c, const float2 *E, const float2 *S0, const float2 *V, const float2 *Mprev,
                            float2 *M, double *out) {
    const int nb = (c->n + TD_PIX - 1) / TD_PIX;
    const size_t smem = (size_t)(TD_PIX + 1) * c->q * sizeof(float2);
    double *part = c->d_mscal + 3 * c->q;
    prof_begin(c, KID_MEC_TDFT);
    k_tdft_fwd<<<nb, 256, smem, c->stream>>>(E, S0, V, Mprev, c->d_twq, c->n, c->q, c->mec_w, V != nullptr,
                                             Mprev != nullptr, M, part);
    k_tdft_finish<<<1, 256, 0, c->stream>>>(part, nb, out);
    prof_end(c, KID_MEC_TDFT);
    return cudaGetLastError();
}

cudaError_t launch_tdft_inv(lrccs_ctx *c, const float2 *M, float omega, float2 *E) {
    const int nb = (c->n + TD_PIX - 1) / TD_PIX;
    const size_t smem = (size_t)(TD_PIX + 1) * c->q * sizeof(float2);
    prof_begin(c, KID_MEC_TDFT);
    k_tdft_inv<<<nb, 256, smem, c->stream>>>(M, c->d_twq, c->n, c->q, c->mec_w, omega, E);
    prof_end(c, KID_MEC_TDFT);
    return cudaGetLastError();
}

// Scratch of the reductions: 3 q FP64 scalars, then max(G q', 3 ceil(n / TD_PIX)) partials.
size_t mec_scal_count(int n, int q, int w) {
    const int nch = (q + w - 1) / w;
    const size_t a = (size_t)MEC_G * nch * w, b = (size_t)3 * ((n + TD_PIX - 1) / TD_PIX);
    return (size_t)3 * q + (a > b ? a : b) + 8;
}
