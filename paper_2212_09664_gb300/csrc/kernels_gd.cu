// kernels_gd.cu -- the GD step of Alg. 2 and its QR re-orthonormalisation as
// one cooperative kernel (one block per SM, every block resident):
//
//   phase 1  grad = Gk - Z B^H  (Gk = sum_j conj(d_j) F^H K_j from the adjoint
//            transforms, Z B^H from k_zb), partial sums of grad^H grad,
//            U^H grad, U^H U
//   -------  grid reduction; every block: eta = eta_c / ||grad||_2 (t = 1),
//            G1 = (U - eta grad)^H (U - eta grad)
//                = U^H U - eta (U^H grad + grad^H U) + eta^2 grad^H grad,
//            G1 = R1^H R1 (Cholesky), R1^{-1}
//   phase 2  U_{t+1} = (U - eta grad) R1^{-1}  (the QR step of Alg. 2 as
//            Cholesky QR), and per block the partial sums of the next
//            B-step's right-hand sides h = U_{t+1}^H Z (the solve adds the
//            blocks' rows in order); the last block out forms SD(U_t, U_{t+1})
//            from U_t^H U_{t+1} = (U^H U - eta U^H grad) R1^{-1}.
//
// G1 is formed from the exact U^H U of the current (FP32) iterate, so each
// iteration removes the loss of orthogonality of the previous one; with
// ||eta grad|| <= eta_c-sized steps G1 is well conditioned and one Cholesky
// QR pass leaves U_{t+1} orthonormal to FP32 rounding.
//
// In init mode the same kernel orthonormalises the given U+ (G1 = U+^H U+)
// and forms the first right-hand sides U_0^H Z.
// A block's pixel range stays in shared memory across the phases when it
// fits; otherwise each phase re-stages it in chunks.
//
// Z B^H depends only on the B-step's result, so its own kernel k_zb forms it
// while the adjoint transforms run (a parallel branch of the iteration).
//
// Partial sums are FP32 within a block and FP64 across blocks, reduced in a
// fixed order (deterministic).  The grid barriers spin on a global counter
// with an iteration limit: a barrier that gives up sets ST_TIMEOUT and the
// kernel runs to completion with that status raised.
#include <math.h>

#include "common.cuh"
#include "internal.h"

#define RMAXC 16   // compile-time bound on the rank
#define NTG 512    // threads per block

struct GdArgs {
    const float2 *Gk;   // n x r   sum_j conj(d_j) F^H K_j (iteration mode)
    const float2 *ZB;   // n x r   Z B^H (iteration mode)
    const float2 *Z;    // n x q   A_k^H y_k, row-major (i q + k)
    float2 *hpart;      // G x q r partial sums of h = U_{t+1}^H Z (row b: block b)
    float2 *U;          // n x r   U_t in, U_{t+1} out
    float2 *Uprev;      // n x r   receives U_t (iteration mode)
    const float2 *Up;   // n x r   U+ (init mode)
    float2 *Gr;         // n x r   receives the gradient (iteration mode)
    float2 *part;       // G x len partial sums
    double2 *tot;       // len totals (FP64)
    double *scal;       // SC_* scalars
    unsigned int *bar;  // [0] barrier arrivals, [1] exit count
    unsigned int *status;
    int n, r, q, zs, chunk, resident, mode;
    double eta_c;
    double eta_scale0, eta_decay;   // variable step size: eta_t = eta eta_scale0 eta_decay^k
    long long *ts;             // NULL, or GD_NTS clock64() stamps per block (phase timing)
    unsigned int spin_limit;   // polls before a grid barrier gives up (2^24 normally)
    unsigned int bar_skew;     // extra arrivals a barrier waits for (0; 1 only for the timeout test)
};

// Phase timing (measurement support): thread 0 of every block stamps clock64()
// at 9 points of the kernel, and the global timer (ns) at its entry and exit,
// when a.ts is set.
#define GD_NTS 11
#define GD_TS(i)                                                                    \
    do {                                                                            \
        if (a.ts && threadIdx.x == 0) a.ts[(size_t)blockIdx.x * GD_NTS + (i)] = clock64(); \
    } while (0)
#define GD_GT(i)                                                                    \
    do {                                                                            \
        if (a.ts && threadIdx.x == 0) {                                             \
            unsigned long long g_;                                                  \
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g_));                  \
            a.ts[(size_t)blockIdx.x * GD_NTS + (i)] = (long long)g_;                \
        }                                                                           \
    } while (0)

// ---------------------------------------------------------------- grid-wide steps

// grid_sync (common.cuh) is the grid-wide barrier of this cooperative kernel.

// Block b reduces entries e = b, b + G, b + 2G, ... (< len) of the G partial
// rows part[g len + e], four entries at a time (128 threads each), into FP64
// totals: per thread in g order, then a fixed shuffle tree, then the warps in
// order.
static __device__ void grid_reduce(const float2 *part, int len, double2 *tot) {
    __shared__ float4 s_w[NTG / 32];   // per warp: (re.hi, re.lo, im.hi, im.lo)
    const int G = gridDim.x, l128 = threadIdx.x & 127, slot = threadIdx.x >> 7;
    for (int j0 = 0; (int)blockIdx.x + G * j0 < len; j0 += NTG / 128) {
        const int e = blockIdx.x + G * (j0 + slot);
        fsum2 re = {0.f, 0.f}, im = {0.f, 0.f};
        if (e < len)
            for (int g = l128; g < G; g += 128) {
                const float2 v = __ldcg(part + (size_t)g * len + e);
                fsum_add(re, v.x);
                fsum_add(im, v.y);
            }
        re = warp_fsum2(re);
        im = warp_fsum2(im);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = make_float4(re.hi, re.lo, im.hi, im.lo);
        __syncthreads();
        if (l128 == 0 && e < len) {
            float4 w = s_w[slot * 4];
            fsum2 R = {w.x, w.y}, I = {w.z, w.w};
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                w = s_w[slot * 4 + k];
                R = fsum_pair(R, fsum2{w.x, w.y});
                I = fsum_pair(I, fsum2{w.z, w.w});
            }
            tot[e] = make_double2((double)R.hi + (double)R.lo, (double)I.hi + (double)I.lo);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- block helpers

// Copy `rows` rows of `cols` complex values (global stride ss, shared stride
// ds) with cp.async, 16 bytes per copy when everything is 16-byte aligned.
static __device__ void stage_rows(float2 *dst, int ds, const float2 *src, int ss, int rows, int cols) {
    if ((((uintptr_t)src | smem_u32(dst)) & 15) == 0 && ((ss | ds | cols) & 1) == 0) {
        const int h = cols >> 1;
        if (h <= (int)blockDim.x) {   // fixed (piece, row-step) mapping: no per-copy division
            const int c2 = threadIdx.x % h, i0 = threadIdx.x / h, step = blockDim.x / h;
            if (i0 < step)
                for (int i = i0; i < rows; i += step) cp_async16(dst + i * ds + 2 * c2, src + (size_t)i * ss + 2 * c2);
            return;
        }
        for (int e = threadIdx.x; e < rows * h; e += blockDim.x) {
            const int i = e / h, c2 = e - i * h;
            cp_async16(dst + i * ds + 2 * c2, src + (size_t)i * ss + 2 * c2);
        }
    } else {
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int i = e / cols, c = e - i * cols;
            cp_async8(dst + i * ds + c, src + (size_t)i * ss + c);
        }
    }
}

// Rinv = (L^H)^{-1} for the lower-triangular L of warp_chol32 (row-major R x R,
// invd = 1 / diag), by one warp: lane j forms column j of X = L^{-1} by
// forward substitution in registers (L read by broadcast), then row j of
// Rinv = X^H (upper triangular).
template <int R>
static __device__ void warp_rinv(const float2 *L, const float *invd, float2 *Rinv) {
    const int j = threadIdx.x & 31;
    float2 x[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        float2 acc = make_float2(i == j ? 1.f : 0.f, 0.f);
#pragma unroll
        for (int m = 0; m < i; ++m) acc = csub(acc, cmul(L[i * R + m], x[m]));
        x[i] = cscale(acc, invd[i]);   // zero for i < j
    }
    if (j < R) {
#pragma unroll
        for (int i = 0; i < R; ++i) Rinv[j * R + i] = i >= j ? cconj(x[i]) : make_float2(0.f, 0.f);
    }
    __syncwarp();
}

// 2 x 2 tile of a cross-Gram: acc[2 i + j] += sum_ii conj(X[ii][x_i]) Y[ii][y_j].
struct Tile {
    const float2 *X, *Y;
    int xs, ys, x0, x1, y0, y1;
};
static __device__ void tile_accumulate(const Tile &g, float2 (&acc)[4], int s, int S, int cn) {
#pragma unroll 4
    for (int ii = s; ii < cn; ii += S) {
        const float2 p0 = g.X[ii * g.xs + g.x0], p1 = g.X[ii * g.xs + g.x1];
        const float2 q0 = g.Y[ii * g.ys + g.y0], q1 = g.Y[ii * g.ys + g.y1];
        cfmac(acc[0], p0, q0);
        cfmac(acc[1], p0, q1);
        cfmac(acc[2], p1, q0);
        cfmac(acc[3], p1, q1);
    }
}

// Combine the slices of up to two tile items per thread (item w = t + u NTG,
// tile w mod T, slice w / T) and write entry m of tile w2 to
// part[blockIdx.x * ld + out(w2, m)] (skipped when out < 0).  One round when
// the scratch scr (cap complex values) holds all four entries of every item,
// else one round per entry through s_red2 (2 NTG values).
template <class OUT>
static __device__ void tiles_write(const float2 (&acc)[2][4], int T, int S, float2 *scr, int cap, float2 *s_red2,
                                   float2 *part, int ld, OUT out) {
    const int W = S * T;
    __syncthreads();
    if (cap >= 4 * W) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int w = threadIdx.x + u * NTG;
            if (w < W) {
#pragma unroll
                for (int m = 0; m < 4; ++m) scr[m * W + w] = acc[u][m];
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < 4 * T; it += NTG) {
            const int m = it / T, w2 = it - m * T;
            const int o = out(w2, m);
            if (o >= 0) {
                float2 sum = make_float2(0.f, 0.f);
                for (int ss = 0; ss < S; ++ss) sum = cadd(sum, scr[m * W + ss * T + w2]);
                part[(size_t)blockIdx.x * ld + o] = sum;
            }
        }
        return;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int w = threadIdx.x + u * NTG;
            if (w < W) s_red2[w] = acc[u][m];
        }
        __syncthreads();
        for (int w2 = threadIdx.x; w2 < T; w2 += NTG) {
            const int o = out(w2, m);
            if (o >= 0) {
                float2 sum = make_float2(0.f, 0.f);
                for (int ss = 0; ss < S; ++ss) sum = cadd(sum, s_red2[ss * T + w2]);
                part[(size_t)blockIdx.x * ld + o] = sum;
            }
        }
    }
}

// ---------------------------------------------------------------- the kernel

template <int R>
__global__ void __launch_bounds__(NTG, 1) k_gdqr(GdArgs a) {
    GD_GT(9);
    extern __shared__ __align__(16) float2 smem[];
    constexpr int r = R;
    const int q = a.q, zs = a.zs, chunk = a.chunk;
    float2 *s_u = smem;                 // chunk * r : U_t (iteration) or U+ (init)
    float2 *s_a = s_u + chunk * r;      // chunk * r : Gk, grad, then U_{t+1}
    float2 *s_w = s_a + chunk * r;      // chunk * r : Z B^H, then U - eta grad
    float2 *s_z = s_w + chunk * r;      // chunk * zs: Z (for h = U_{t+1}^H Z)
    __shared__ float2 sL[R * R];
    __shared__ float2 sR[R * R];
    __shared__ float sinv[R];
    __shared__ float2 s_tot[2 * (R * (R + 1) / 2) + R * R];
    __shared__ float2 s_red2[2 * NTG];
    __shared__ float s_c[RMAXC], s_s[RMAXC];
    __shared__ float2 s_e[RMAXC];
    __shared__ int s_cnt, s_flag;
    __shared__ float s_eta;
    const int t = threadIdx.x, G = gridDim.x;
    const int np = r * (r + 1) / 2, rr = r * r, tr = (r + 1) >> 1;
    const int per = (a.n + G - 1) / G;
    const int i0 = min(a.n, (int)blockIdx.x * per), i1 = min(a.n, i0 + per);
    const bool iter = a.mode == 1;
    // eta as it stands at launch; block 0 updates the device copy only after
    // every block has passed the first barrier (so after every block read it)
    const double eta_in = a.scal[SC_ETA];
    const bool eta_set = a.scal[SC_ETASET] != 0.0;
    const double tcnt = eta_set ? a.scal[SC_TCNT] : 0.0;   // iterations since eta was set

    // ------------------------------------------------ phase 1: gradient and Gram partial sums
    // tiles: [grad^H grad (upper tiles) | U^H grad (all) | U^H U (upper tiles)], init: [U+^H U+]
    const int th = tr * (tr + 1) / 2;
    const int T1 = iter ? 2 * th + tr * tr : th;
    const int len1 = iter ? 2 * np + rr : np;
    const int S1 = max(1, NTG / T1);
    auto tile1 = [&](int w, int &kind, int &A, int &Bt) {
        if (!iter) {
            kind = 2;
            pair_of(w, tr, A, Bt);
        } else if (w < th) {
            kind = 0;
            pair_of(w, tr, A, Bt);
        } else if (w < th + tr * tr) {
            kind = 1;
            A = (w - th) / tr;
            Bt = (w - th) - A * tr;
        } else {
            kind = 2;
            pair_of(w - th - tr * tr, tr, A, Bt);
        }
    };
    Tile g1[2];
    int sl1[2];
    float2 acc[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int w = t + u * NTG;
        sl1[u] = w < S1 * T1 ? w / T1 : S1;   // S1 marks an idle item
        int kind = 0, A = 0, Bt = 0;
        if (w < S1 * T1) tile1(w % T1, kind, A, Bt);
        g1[u].X = kind == 0 ? s_a : s_u;
        g1[u].Y = kind == 2 ? s_u : s_a;
        g1[u].xs = g1[u].ys = r;
        g1[u].x0 = 2 * A;
        g1[u].x1 = min(2 * A + 1, r - 1);
        g1[u].y0 = 2 * Bt;
        g1[u].y1 = min(2 * Bt + 1, r - 1);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[u][m] = make_float2(0.f, 0.f);
    }
    GD_TS(0);
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        __syncthreads();
        if (iter) {
            stage_rows(s_a, r, a.Gk + (size_t)c0 * r, r, cn, r);
            stage_rows(s_u, r, a.U + (size_t)c0 * r, r, cn, r);
            stage_rows(s_w, r, a.ZB + (size_t)c0 * r, r, cn, r);
        } else {
            stage_rows(s_u, r, a.Up + (size_t)c0 * r, r, cn, r);
        }
        cp_async_commit();
        if (a.resident) {   // Z for phase 2 streams in behind phase 1
            stage_rows(s_z, zs, a.Z + (size_t)c0 * q, q, cn, q);
            cp_async_commit();
            cp_async_wait_1();
        } else {
            cp_async_wait();
        }
        __syncthreads();
        if (c0 == i0) GD_TS(1);
        if (iter) {   // grad = Gk - Z B^H
            for (int e = t; e < cn * r; e += NTG) {
                const float2 g = csub(s_a[e], s_w[e]);
                s_a[e] = g;
                a.Gr[(size_t)c0 * r + e] = g;
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (sl1[u] < S1) tile_accumulate(g1[u], acc[u], sl1[u], S1, cn);
    }
    GD_TS(2);
    // partial row: [grad^H grad pairs (np) | U^H grad (rr) | U^H U pairs (np)], init: [U+^H U+ pairs]
    tiles_write(acc, T1, S1, s_w, chunk * r, s_red2, a.part, len1, [&](int w, int m) {
        int kind, A, Bt;
        tile1(w, kind, A, Bt);
        const int x = 2 * A + (m >> 1), y = 2 * Bt + (m & 1);
        if (x >= r || y >= r) return -1;
        if (kind == 1) return np + x * r + y;
        if (x > y) return -1;
        return (kind == 2 && iter ? np + rr : 0) + pair_index(x, y, r);
    });
    GD_TS(3);
    grid_sync(a.bar, 1, a.status, a.spin_limit, a.bar_skew, ST_TIMEOUT);
    GD_TS(4);
    grid_reduce(a.part, len1, a.tot);
    GD_TS(5);
    grid_sync(a.bar, 2, a.status, a.spin_limit, a.bar_skew, ST_TIMEOUT);
    GD_TS(6);
    for (int e = t; e < len1; e += NTG) {
        const double2 v = __ldcg(a.tot + e);
        s_tot[e] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();

    // ------------------------------------------------ G1 = R1^H R1 and R1^{-1} (every block)
    if (iter) {
        const float2 *A1 = s_tot, *A2 = s_tot + np, *A3 = s_tot + np + rr;
        if (t == 0) s_eta = (float)eta_in;
        if (!eta_set) {
            // ||grad||_2^2 = lambda_max(grad^H grad) (Alg. 2, t = 1), FP32 Jacobi
            for (int p = t; p < np; p += NTG) {
                int x, y;
                pair_of(p, r, x, y);
                sR[x * r + y] = A1[p];
                sR[y * r + x] = cconj(A1[p]);
            }
            __syncthreads();
            block_jacobi(sR, r, r, nullptr, 0, s_c, s_s, s_e, &s_cnt, 30);
            if (t == 0) {
                float lmax = 0.f;
                for (int x = 0; x < r; ++x) lmax = fmaxf(lmax, sR[x * r + x].x);
                const double gn = sqrt((double)lmax);
                const double eta = gn > 0.0 ? a.eta_c / gn : 0.0;
                s_eta = (float)eta;
                if (blockIdx.x == 0) {
                    a.scal[SC_GNORM] = gn;
                    a.scal[SC_ETA] = eta;
                    a.scal[SC_ETASET] = 1.0;
                }
            }
        }
        // the step of this iteration (constant unless a schedule is set), and
        // the schedule's counter for the next one (every block has read it)
        if (t == 0) {
            if (a.eta_scale0 != 1.0 || a.eta_decay != 1.0)
                s_eta = (float)((double)s_eta * a.eta_scale0 * pow(a.eta_decay, tcnt));
            if (blockIdx.x == 0) a.scal[SC_TCNT] = tcnt + 1.0;
        }
        __syncthreads();
        const float eta = s_eta, eta2 = s_eta * s_eta;
        for (int e = t; e < rr; e += NTG) {
            const int x = e / r, y = e - x * r;
            const int p = x <= y ? pair_index(x, y, r) : pair_index(y, x, r);
            const float sg = x <= y ? 1.f : -1.f;   // lower half: conjugate of the stored pair
            const float x2r = A2[x * r + y].x + A2[y * r + x].x;
            const float x2i = A2[x * r + y].y - A2[y * r + x].y;
            sL[e] = make_float2(A3[p].x - eta * x2r + eta2 * A1[p].x, sg * A3[p].y - eta * x2i + eta2 * sg * A1[p].y);
        }
    } else {
        for (int e = t; e < rr; e += NTG) {
            const int x = e / r, y = e - x * r;
            const int p = x <= y ? pair_index(x, y, r) : pair_index(y, x, r);
            sL[e] = x <= y ? s_tot[p] : cconj(s_tot[p]);
        }
    }
    __syncthreads();
    // G1 = L L^H and R1^{-1} = (L^H)^{-1} by the first warp in registers (the
    // other warps wait at the barrier below)
    if (t < 32) {
        if (!warp_chol32<R>(sL, R, sinv)) {
            if (t == 0 && blockIdx.x == 0) atomicOr(a.status, (unsigned)ST_NOT_SPD_QR);
            for (int e = t; e < rr; e += 32) sL[e] = make_float2(e / r == e % r ? 1.f : 0.f, 0.f);
            if (t < r) sinv[t] = 1.f;
            __syncwarp();
        }
        warp_rinv<R>(sL, sinv, sR);
    }
    __syncthreads();
    GD_TS(7);
    const float etaf = iter ? s_eta : 0.f;

    // ------------------------------------------------ phase 2: U_{t+1} = (U - eta grad) R1^{-1}
    // and the partial sums of h = U_{t+1}^H Z over the block's pixels, thread
    // (frame pair kp, slice hs) holding all R columns for frames 2 kp, 2 kp + 1
    const int tq = (q + 1) >> 1;
    const int Sh = max(1, NTG / tq), Hth = tq * Sh;
    const bool hthr = t < Hth;
    const int hk = 2 * (t % tq), hs = t / tq;
    float2 pv[2 * R];
#pragma unroll
    for (int v = 0; v < 2 * R; ++v) pv[v] = make_float2(0.f, 0.f);
    for (int c0 = i0; c0 < i1; c0 += chunk) {
        const int cn = min(chunk, i1 - c0);
        if (!a.resident) {
            __syncthreads();
            if (iter) {
                stage_rows(s_u, r, a.U + (size_t)c0 * r, r, cn, r);
                stage_rows(s_a, r, a.Gr + (size_t)c0 * r, r, cn, r);
            } else {
                stage_rows(s_u, r, a.Up + (size_t)c0 * r, r, cn, r);
            }
            stage_rows(s_z, zs, a.Z + (size_t)c0 * q, q, cn, q);
            cp_async_commit();
        }
        cp_async_wait();
        __syncthreads();
        for (int e = t; e < cn * r; e += NTG) s_w[e] = iter ? csub(s_u[e], cscale(s_a[e], etaf)) : s_u[e];
        __syncthreads();
        for (int e = t; e < cn * r; e += NTG) {
            const int ii = e / r, l = e - ii * r;
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < R; ++m)
                if (m <= l) cfma(v, s_w[ii * r + m], sR[m * r + l]);
            s_a[e] = v;
            a.U[(size_t)c0 * r + e] = v;
            if (iter) a.Uprev[(size_t)c0 * r + e] = s_u[e];
        }
        __syncthreads();
        if (hthr) {
#pragma unroll(R <= 12 ? 2 : 1)
            for (int ii = hs; ii < cn; ii += Sh) {
                const float4 z = *(const float4 *)(s_z + ii * zs + hk);   // Z[k], Z[k+1] (pad column when k+1 = q)
                const float2 z0 = make_float2(z.x, z.y), z1 = make_float2(z.z, z.w);
                if constexpr ((R & 1) == 0) {   // U_{t+1} row in 16-byte pairs (r even: rows 16-byte aligned)
                    const float4 *u4 = (const float4 *)(s_a + ii * r);
#pragma unroll
                    for (int l2 = 0; l2 < R / 2; ++l2) {
                        const float4 uu = u4[l2];
                        const float2 ua = make_float2(uu.x, uu.y), ub = make_float2(uu.z, uu.w);
                        cfmac(pv[2 * l2], ua, z0);
                        cfmac(pv[R + 2 * l2], ua, z1);
                        cfmac(pv[2 * l2 + 1], ub, z0);
                        cfmac(pv[R + 2 * l2 + 1], ub, z1);
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < R; ++l) {
                        const float2 u = s_a[ii * r + l];
                        cfmac(pv[l], u, z0);
                        cfmac(pv[R + l], u, z1);
                    }
                }
            }
        }
    }
    // the block's row of h partial sums, hpart[b][k r + l], slices added in
    // order, V values per thread per round (s_w and s_z are free now)
    {
        const int cap2 = chunk * (r + zs);
        float2 *scr = cap2 >= 2 * NTG ? s_w : s_red2;
        const int V = max(2, min(2 * R, ((cap2 >= 2 * NTG ? cap2 : 2 * NTG) / NTG) & ~1));
        float2 *hrow = a.hpart + (size_t)blockIdx.x * q * r;
        for (int v0 = 0; v0 < 2 * R; v0 += V) {
            __syncthreads();
            if (hthr) {
#pragma unroll
                for (int v = 0; v < 2 * R; ++v)
                    if (v >= v0 && v < v0 + V) scr[(v - v0) * NTG + t] = pv[v];
            }
            __syncthreads();
            const int vn = min(V, 2 * R - v0);
            for (int w = t; w < vn * tq; w += NTG) {
                const int dv = w / tq, kp = w - dv * tq, v = v0 + dv;
                const int k = 2 * kp + v / R, l = v % R;
                if (k < q) {
                    float2 sum = make_float2(0.f, 0.f);
                    for (int ss = 0; ss < Sh; ++ss) sum = cadd(sum, scr[dv * NTG + ss * tq + kp]);
                    hrow[k * r + l] = sum;
                }
            }
        }
    }
    GD_TS(8);
    // the last block out: SD(U_t, U_{t+1})^2 = r - ||U_t^H U_{t+1}||_F^2 with
    // U_t^H U_{t+1} = (U_t^H U_t - eta U_t^H grad) R1^{-1} from the totals (no
    // second reduction; thread x r + y forms entry (x, y)), and the barrier
    // counters back to zero (every block is past its last barrier)
    __syncthreads();
    if (t == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(a.bar + 1, 1u);
        s_flag = prev == (unsigned)G - 1;
    }
    __syncthreads();
    if (!s_flag) {
        GD_GT(10);
        return;
    }
    double sq = 0.0;
    if (iter && t < rr) {
        const float2 *A2 = s_tot + np, *A3 = s_tot + np + rr;
        const int x = t / r, y = t - x * r;
        float2 mv = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if (m <= y) {
                const float2 uu = x <= m ? A3[pair_index(x, m, r)] : cconj(A3[pair_index(m, x, r)]);
                cfma(mv, csub(uu, cscale(A2[x * r + m], etaf)), sR[m * r + y]);
            }
        }
        sq = (double)mv.x * mv.x + (double)mv.y * mv.y;
    }
    // block sum in a fixed order: warps, then warp 0 over the warp sums
    __shared__ double s_sq[NTG / 32];
    sq = warp_sum_d(sq);
    if ((t & 31) == 0) s_sq[t >> 5] = sq;
    __syncthreads();
    if (t < 32) {
        double sum = t < NTG / 32 ? s_sq[t] : 0.0;
        sum = warp_sum_d(sum);
        if (t == 0) {
            if (iter) {
                const double sd2 = (double)r - sum;
                a.scal[SC_SD] = sqrt(sd2 > 0.0 ? sd2 : 0.0);
            }
            a.bar[0] = 0u;
            a.bar[1] = 0u;
        }
    }
    GD_GT(10);
}

// ---------------------------------------------------------------- Z contractions

// Z B^H (n x r): ZB[i][l] = sum_k Z[i][k] conj(B[k][l]), the data term of the
// gradient grad = Gk - Z B^H (Alg. 2).  Block = ZB_PIX pixels, thread = (pixel,
// half of the l range); the pixels' Z rows are staged with an odd row stride
// (conflict-free 8-byte loads across pixels), B is read by broadcast.
#define ZB_PIX 128
template <int R>
__global__ void __launch_bounds__(256) k_zb(const float2 *__restrict__ Z, const float2 *__restrict__ B, int n, int q,
                                            float2 *__restrict__ ZB) {
    extern __shared__ __align__(16) float2 smem[];
    constexpr int RH = (R + 1) / 2;
    const int zs = q | 1;
    float2 *s_z = smem;               // ZB_PIX * zs
    float2 *s_b = s_z + ZB_PIX * zs;  // q * R
    const int i0 = blockIdx.x * ZB_PIX, cn = min(ZB_PIX, n - i0);
    for (int e = threadIdx.x; e < cn * q; e += blockDim.x) {
        const int ii = e / q, k = e - ii * q;
        cp_async8(s_z + ii * zs + k, Z + (size_t)i0 * q + e);
    }
    for (int e = threadIdx.x; e < q * R; e += blockDim.x) cp_async8(s_b + e, B + e);
    cp_async_commit();
    cp_async_wait();
    __syncthreads();
    const int p = threadIdx.x & (ZB_PIX - 1), h = threadIdx.x / ZB_PIX;
    if (p >= cn) return;
    const int l0 = h * RH, nl = min(RH, R - l0);
    float2 acc[RH];
#pragma unroll
    for (int j = 0; j < RH; ++j) acc[j] = make_float2(0.f, 0.f);
    const float2 *zr = s_z + p * zs;
#pragma unroll 4
    for (int k = 0; k < q; ++k) {
        const float2 z = zr[k];
#pragma unroll
        for (int j = 0; j < RH; ++j)
            if (j < nl) cfmac(acc[j], s_b[k * R + l0 + j], z);   // conj(b) z
    }
#pragma unroll
    for (int j = 0; j < RH; ++j)
        if (j < nl) ZB[(size_t)(i0 + p) * R + l0 + j] = acc[j];
}

// ---------------------------------------------------------------- launcher

typedef void (*gd_kernel_t)(GdArgs);
static const gd_kernel_t kGd[RMAXC] = {k_gdqr<1>,  k_gdqr<2>,  k_gdqr<3>,  k_gdqr<4>,  k_gdqr<5>,  k_gdqr<6>,
                                       k_gdqr<7>,  k_gdqr<8>,  k_gdqr<9>,  k_gdqr<10>, k_gdqr<11>, k_gdqr<12>,
                                       k_gdqr<13>, k_gdqr<14>, k_gdqr<15>, k_gdqr<16>};
static int g_gd_static_smem[RMAXC];

cudaError_t configure_kernels_gd(int max_smem) {
    for (int i = 0; i < RMAXC; ++i) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kGd[i]);
        if (e != cudaSuccess) return e;
        g_gd_static_smem[i] = (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(kGd[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Z row stride in shared memory: q rounded up to 2 mod 4 complex values, so
// that 16-byte loads of consecutive pixels' rows hit distinct banks.
static int z_stride(int q) { return ((q + 1) | 3) - 1; }

cudaError_t launch_gdqr(lrccs_ctx *c, int mode) {
    const int r = c->r, q = c->q, G = c->gd_grid;
    if (r < 1 || r > RMAXC) return cudaErrorInvalidValue;
    const int zs = z_stride(q);
    const int per = (c->n + G - 1) / G;
    const size_t bpp = (size_t)(3 * r + zs) * sizeof(float2);
    const size_t avail = (size_t)(c->dev_smem_optin - g_gd_static_smem[r - 1]);
    int chunk = (int)(avail / bpp) & ~1;
    chunk = min(chunk, 512);
    chunk = min(chunk, (per + 1) & ~1);
    if (chunk < 2) return cudaErrorInvalidConfiguration;
    GdArgs a;
    a.Gk = c->d_Up;
    a.ZB = c->d_ZB;
    a.Z = c->d_Z;
    a.hpart = c->d_hpart;
    a.U = c->d_U;
    a.Uprev = c->d_Uprev;
    a.Up = c->d_Up;
    a.Gr = c->d_G;
    a.part = c->d_gpart;
    a.tot = c->d_tot;
    a.scal = c->d_scal;
    a.bar = c->d_counters + CNT_BAR;
    a.status = c->d_status;
    a.n = c->n;
    a.r = r;
    a.q = q;
    a.zs = zs;
    a.chunk = chunk;
    a.resident = chunk >= per ? 1 : 0;
    a.mode = mode;
    a.eta_c = c->prm.eta_c;
    a.eta_scale0 = c->prm.eta_scale0 > 0.0 ? c->prm.eta_scale0 : 1.0;
    a.eta_decay = c->prm.eta_decay > 0.0 ? c->prm.eta_decay : 1.0;
    a.spin_limit = 1u << 24;
    a.bar_skew = 0;
    a.ts = mode == 1 ? c->d_gdts : nullptr;   // also in captured iterations (phase timing on)
    if (c->test_timeout && !c->capturing) {   // lrccs_test_wait_timeout: this launch only
        a.spin_limit = 1u << 16;
        a.bar_skew = 1;
        c->test_timeout = 0;
    }
    void *args[] = {&a};
    const size_t smem = (size_t)chunk * bpp;
    prof_begin(c, KID_GDQR);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kGd[r - 1], dim3(G), dim3(NTG), args, smem, c->stream);
    prof_end(c, KID_GDQR);
    return e;
}

typedef void (*zb_kernel_t)(const float2 *, const float2 *, int, int, float2 *);
#define RANK_TABLE(K) {K<1>, K<2>, K<3>, K<4>, K<5>, K<6>, K<7>, K<8>, K<9>, K<10>, K<11>, K<12>, K<13>, K<14>, K<15>, K<16>}
static const zb_kernel_t kZb[RMAXC] = RANK_TABLE(k_zb);

static size_t zb_smem(int q, int r) { return ((size_t)ZB_PIX * (q | 1) + (size_t)q * r) * sizeof(float2); }
// d_ZB <- Z B^H (the data term of the next gradient), from the current B.
cudaError_t launch_zb(lrccs_ctx *c) {
    const int r = c->r;
    if (r < 1 || r > RMAXC) return cudaErrorInvalidValue;
    prof_begin(c, KID_ZB);
    kZb[r - 1]<<<(c->n + ZB_PIX - 1) / ZB_PIX, 256, zb_smem(c->q, r), c->stream>>>(c->d_Z, c->d_B, c->n, c->q,
                                                                                   c->d_ZB);
    prof_end(c, KID_ZB);
    return cudaGetLastError();
}

cudaError_t configure_kernels_zh(int max_smem) {
    for (int i = 0; i < RMAXC; ++i) {
        const int r = i + 1;
        const size_t a = zb_smem(128, r);   // the largest q
        if ((int)a > max_smem) return cudaErrorInvalidConfiguration;
        cudaError_t e = cudaFuncSetAttribute(kZb[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
