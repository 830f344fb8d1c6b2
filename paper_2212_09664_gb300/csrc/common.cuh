// common.cuh -- complex helpers, the warp-level FFT engine and block reductions
// shared by the liblrccs kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define LRCCS_DEV __device__ __forceinline__

// ---------------------------------------------------------------- complex64

LRCCS_DEV float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// conj(a) * b
LRCCS_DEV float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
LRCCS_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
LRCCS_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
LRCCS_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
LRCCS_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc += a * b
LRCCS_DEV void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
LRCCS_DEV void cfmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
LRCCS_DEV float2 shfl_xor2(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

struct dcomplex { double x, y; };
LRCCS_DEV dcomplex dc(double x, double y) { dcomplex r; r.x = x; r.y = y; return r; }
LRCCS_DEV dcomplex dmul(dcomplex a, dcomplex b) { return dc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
LRCCS_DEV dcomplex dmulc(dcomplex a, dcomplex b) { return dc(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
LRCCS_DEV dcomplex dadd(dcomplex a, dcomplex b) { return dc(a.x + b.x, a.y + b.y); }
LRCCS_DEV dcomplex dsub(dcomplex a, dcomplex b) { return dc(a.x - b.x, a.y - b.y); }

LRCCS_DEV int brev5(int v) { return (int)(__brev((unsigned)v) >> 27); }

// Upper-triangle pair enumeration of an r x r Hermitian matrix: p -> (a, b), a <= b.
LRCCS_DEV void pair_of(int p, int r, int &a, int &b) {
    int aa = 0;
    int rem = p;
    while (rem >= r - aa) { rem -= r - aa; ++aa; }
    a = aa;
    b = aa + rem;
}
LRCCS_DEV int pair_index(int a, int b, int r) {  // a <= b
    return a * r - (a * (a - 1)) / 2 + (b - a);
}

// Load the twiddle table of length N into shared memory.
// |v|^2 in FP64 without contraction: the truncation decision |y|^2 <= gamma of
// the spectral initialisation is taken on exactly the squares an FP64
// reference forms.
LRCCS_DEV double abs2_rn(float2 v) {
    return __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y));
}

LRCCS_DEV void load_twiddles(float2 *s_tw, const float2 *g_tw, int N) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) s_tw[t] = g_tw[t];
}

// ---------------------------------------------------------------- grid reductions
//
// "Last block" pattern: each block writes its partial, fences, and increments a
// counter; the block that sees count == gridDim-1 reduces all partials in a
// fixed order (deterministic) and resets the counter for the next launch.
LRCCS_DEV bool last_block_arrive(unsigned int *counter) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nblk - 1);
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// ---------------------------------------------------------------- Hermitian eigensolver

// Parallel cyclic Jacobi for an n x n Hermitian matrix A in shared memory
// (all threads of the block call it).  Rounds follow the circle ordering, so
// the n/2 rotations of a round touch disjoint index pairs.  Each rotation
// removes the phase of a_pq and applies the real 2x2 Jacobi rotation:
// G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]], A <- G^H A G, V <- V G.
// V (ldv columns, may be global memory) is updated when non-null.
// A rotation is skipped when |a_pq| <= rel_tol sqrt(|a_pp a_qq|) or |a_pq| <= abs_tol,
// or when both |a_pp| and |a_qq| are below tail_tol (a rotation between two
// such indices only mixes columns p and q of V: when every wanted eigenvalue
// is above tail_tol, the wanted eigenvectors converge without them);
// the sweeps stop when a whole sweep skips every rotation.
__device__ inline void block_jacobi(float2 *A, int n, int lda, float2 *V, int ldv, float *s_c, float *s_s, float2 *s_e,
                             int *s_cnt, int max_sweeps, float abs_tol = 0.f, float rel_tol = 1e-7f,
                             float tail_tol = 0.f) {
    const int n2 = n + (n & 1);
    const int npair = n2 / 2;
    int sh = 0;                             // column index stride 2^sh >= n (no division per task)
    while ((1 << sh) < n) ++sh;
    const int mmask = (1 << sh) - 1;
    int psh = 0;                            // pair index stride 2^psh >= npair
    while ((1 << psh) < npair) ++psh;
    const int pmask = (1 << psh) - 1;
    __shared__ short s_pp[64], s_qq[64];   // the pairs of the current round
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *s_cnt = 0;
        __syncthreads();
        for (int rnd = 0; rnd < n2 - 1; ++rnd) {
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                int p, qq;
                if (i == 0) { p = rnd; qq = n2 - 1; }
                else { p = (rnd + i) % (n2 - 1); qq = (rnd - i + n2 - 1) % (n2 - 1); }
                s_pp[i] = (short)p;
                s_qq[i] = (short)qq;
                float c = 1.f, s = 0.f;
                float2 e = make_float2(1.f, 0.f);
                if (p < n && qq < n) {
                    const float2 apq = A[p * lda + qq];
                    const float b2 = apq.x * apq.x + apq.y * apq.y;
                    const float al = A[p * lda + p].x, ga = A[qq * lda + qq].x;
                    if (b2 > 1e-36f && b2 > abs_tol * abs_tol && b2 > rel_tol * rel_tol * fabsf(al) * fabsf(ga) &&
                        (fabsf(al) >= tail_tol || fabsf(ga) >= tail_tol)) {
                        // the rotation only has to be orthogonal: c = 1 / sqrt(1 + t^2),
                        // s = t c hold to rounding whatever the accuracy of t
                        const float ib = rsqrtf(b2);
                        e = make_float2(apq.x * ib, apq.y * ib);
                        const float tau = (ga - al) * 0.5f * ib;
                        const float t = copysignf(1.f, tau) * __frcp_rn(fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
                        c = rsqrtf(fmaf(t, t, 1.f));
                        s = t * c;
                        *s_cnt = 1;
                    }
                }
                s_c[i] = c;
                s_s[i] = s;
                s_e[i] = e;
            }
            __syncthreads();
            // A <- G^H A G on the 2 x 2 blocks (rows of pair i, columns of
            // pair i2: disjoint, so one pass; the row rotation first, then
            // the column rotation, as two separate passes would), and V <- V G
            const int nab = npair << psh;
            for (int task = threadIdx.x; task < nab + (V ? (npair << sh) : 0); task += blockDim.x) {
                if (task < nab) {
                    const int i = task >> psh, i2 = task & pmask;
                    if (i2 >= npair) continue;
                    const float si = s_s[i], si2 = s_s[i2];
                    if (si == 0.f && si2 == 0.f) continue;
                    const int p = s_pp[i], qq = s_qq[i], p2 = s_pp[i2], q2 = s_qq[i2];
                    const bool r0 = p < n, r1 = qq < n, c0 = p2 < n, c1 = q2 < n;
                    const float2 z = make_float2(0.f, 0.f);
                    float2 a00 = r0 && c0 ? A[p * lda + p2] : z, a01 = r0 && c1 ? A[p * lda + q2] : z;
                    float2 a10 = r1 && c0 ? A[qq * lda + p2] : z, a11 = r1 && c1 ? A[qq * lda + q2] : z;
                    if (si != 0.f) {   // rows p, q of columns p2, q2
                        const float c = s_c[i];
                        const float2 e = s_e[i];
                        float2 eaq = cmul(e, a10);
                        float2 ap = a00;
                        a00 = make_float2(c * ap.x - si * eaq.x, c * ap.y - si * eaq.y);
                        a10 = make_float2(si * ap.x + c * eaq.x, si * ap.y + c * eaq.y);
                        eaq = cmul(e, a11);
                        ap = a01;
                        a01 = make_float2(c * ap.x - si * eaq.x, c * ap.y - si * eaq.y);
                        a11 = make_float2(si * ap.x + c * eaq.x, si * ap.y + c * eaq.y);
                    }
                    if (si2 != 0.f) {   // columns p2, q2 of rows p, q
                        const float c = s_c[i2];
                        const float2 eh = cconj(s_e[i2]);
                        float2 e2 = cmul(eh, a01);
                        float2 ap = a00;
                        a00 = make_float2(c * ap.x - si2 * e2.x, c * ap.y - si2 * e2.y);
                        a01 = make_float2(si2 * ap.x + c * e2.x, si2 * ap.y + c * e2.y);
                        e2 = cmul(eh, a11);
                        ap = a10;
                        a10 = make_float2(c * ap.x - si2 * e2.x, c * ap.y - si2 * e2.y);
                        a11 = make_float2(si2 * ap.x + c * e2.x, si2 * ap.y + c * e2.y);
                    }
                    if (r0 && c0) A[p * lda + p2] = a00;
                    if (r0 && c1) A[p * lda + q2] = a01;
                    if (r1 && c0) A[qq * lda + p2] = a10;
                    if (r1 && c1) A[qq * lda + q2] = a11;
                } else {
                    const int tv = task - nab, i = tv >> sh, m = tv & mmask;
                    if (m >= n || s_s[i] == 0.f) continue;
                    const int p = s_pp[i], qq = s_qq[i];
                    const float c = s_c[i], s = s_s[i];
                    const float2 eh = cconj(s_e[i]);
                    const float2 vp = V[m * ldv + p], vq = V[m * ldv + qq];
                    const float2 e2 = cmul(eh, vq);
                    V[m * ldv + p] = make_float2(c * vp.x - s * e2.x, c * vp.y - s * e2.y);
                    V[m * ldv + qq] = make_float2(s * vp.x + c * e2.x, s * vp.y + c * e2.y);
                }
            }
            __syncthreads();
        }
        if (*s_cnt == 0) break;
        __syncthreads();
    }
    __syncthreads();
}


// Allow a kernel the device's opt-in shared memory per block, minus its static
// shared memory (the launch still requests only what it needs).
template <typename K>
static inline cudaError_t allow_smem(K kernel, int optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
}

// ---------------------------------------------------------------- warp-level FP64 small linear algebra
// For the r x r (r <= 32) Hermitian systems of the B-step and of CholeskyQR2.
// Matrices are FP64 (re, im) pairs, row-major, in shared memory; one full warp
// calls each routine.  GB300's FP64 pipe is narrow, so the work is spread over
// the lanes instead of running on one thread.

LRCCS_DEV double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;  // identical in every lane (each level adds the same two numbers)
}

// In place A = L L^H: the lower triangle of A receives L (real positive
// diagonal).  Returns false (in every lane) if A is not positive definite.
LRCCS_DEV bool warp_cholesky(double *A, int r) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < r; ++c) {
        double part = 0.0;
        if (lane < c) {
            const double ar = A[(c * r + lane) * 2], ai = A[(c * r + lane) * 2 + 1];
            part = ar * ar + ai * ai;
        }
        part = warp_sum_d(part);
        double d = A[(c * r + c) * 2] - part;
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        __syncwarp();
        if (lane > c && lane < r) {
            double vr = A[(lane * r + c) * 2], vi = A[(lane * r + c) * 2 + 1];
            for (int m = 0; m < c; ++m) {  // v -= L[lane][m] conj(L[c][m])
                const double ar = A[(lane * r + m) * 2], ai = A[(lane * r + m) * 2 + 1];
                const double br = A[(c * r + m) * 2], bi = A[(c * r + m) * 2 + 1];
                vr -= ar * br + ai * bi;
                vi -= ai * br - ar * bi;
            }
            A[(lane * r + c) * 2] = vr / d;
            A[(lane * r + c) * 2 + 1] = vi / d;
        }
        __syncwarp();
        if (lane == 0) {
            A[(c * r + c) * 2] = d;
            A[(c * r + c) * 2 + 1] = 0.0;
        }
        __syncwarp();
    }
    return true;
}

// Rinv = (L^H)^{-1} (upper triangular) from the lower factor L in A.
// Li: r * r * 2 doubles of shared scratch.  Lane j computes column j of L^{-1}.
LRCCS_DEV void warp_rinv(const double *A, int r, double *Li, double *Rinv) {
    const int lane = threadIdx.x & 31;
    if (lane < r) {
        const int j = lane;
        for (int i = 0; i < j; ++i) {
            Li[(i * r + j) * 2] = 0.0;
            Li[(i * r + j) * 2 + 1] = 0.0;
        }
        Li[(j * r + j) * 2] = 1.0 / A[(j * r + j) * 2];
        Li[(j * r + j) * 2 + 1] = 0.0;
        for (int i = j + 1; i < r; ++i) {
            double vr = 0.0, vi = 0.0;
            for (int m = j; m < i; ++m) {
                const double ar = A[(i * r + m) * 2], ai = A[(i * r + m) * 2 + 1];
                const double br = Li[(m * r + j) * 2], bi = Li[(m * r + j) * 2 + 1];
                vr += ar * br - ai * bi;
                vi += ar * bi + ai * br;
            }
            const double d = A[(i * r + i) * 2];
            Li[(i * r + j) * 2] = -vr / d;
            Li[(i * r + j) * 2 + 1] = -vi / d;
        }
    }
    __syncwarp();
    for (int e = lane; e < r * r; e += 32) {
        const int a = e / r, b = e - a * r;
        Rinv[e * 2] = Li[(b * r + a) * 2];
        Rinv[e * 2 + 1] = -Li[(b * r + a) * 2 + 1];
    }
    __syncwarp();
}

// Solve L L^H x = h (L lower in A); h and x are r (re, im) pairs in shared memory.
LRCCS_DEV void warp_chol_solve(const double *A, int r, const double *h, double *x) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < r; ++c) {  // L z = h
        double pr = 0.0, pi = 0.0;
        if (lane < c) {
            const double ar = A[(c * r + lane) * 2], ai = A[(c * r + lane) * 2 + 1];
            const double zr = x[2 * lane], zi = x[2 * lane + 1];
            pr = ar * zr - ai * zi;
            pi = ar * zi + ai * zr;
        }
        pr = warp_sum_d(pr);
        pi = warp_sum_d(pi);
        const double d = A[(c * r + c) * 2];
        if (lane == 0) {
            x[2 * c] = (h[2 * c] - pr) / d;
            x[2 * c + 1] = (h[2 * c + 1] - pi) / d;
        }
        __syncwarp();
    }
    for (int c = r - 1; c >= 0; --c) {  // L^H x = z
        double pr = 0.0, pi = 0.0;
        if (lane > c && lane < r) {  // conj(L[lane][c]) x[lane]
            const double ar = A[(lane * r + c) * 2], ai = -A[(lane * r + c) * 2 + 1];
            const double zr = x[2 * lane], zi = x[2 * lane + 1];
            pr = ar * zr - ai * zi;
            pi = ar * zi + ai * zr;
        }
        pr = warp_sum_d(pr);
        pi = warp_sum_d(pi);
        const double d = A[(c * r + c) * 2];
        __syncwarp();
        if (lane == 0) {
            x[2 * c] = (x[2 * c] - pr) / d;
            x[2 * c + 1] = (x[2 * c + 1] - pi) / d;
        }
        __syncwarp();
    }
}

// Compensated FP32 summation (Knuth's two-sum): a (hi, lo) pair carries ~48
// bits, at FP32 speed (an FP64 add is ~14x slower on this GPU).
struct fsum2 {
    float hi, lo;
};
LRCCS_DEV void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
LRCCS_DEV void fsum_add(fsum2 &acc, float x) {
    float s, e;
    two_sum(acc.hi, x, s, e);
    acc.hi = s;
    acc.lo += e;
}
// Warp-wide sum of (hi, lo) pairs, kept as a pair; identical in every lane.
LRCCS_DEV fsum2 warp_fsum2(fsum2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o), ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
        float s, e;
        const bool first = (threadIdx.x & o) == 0;
        two_sum(first ? v.hi : oh, first ? oh : v.hi, s, e);
        v.lo = (first ? v.lo + ol : ol + v.lo) + e;
        v.hi = s;
    }
    return v;
}
// (hi, lo) pair sum a + b (a first)
LRCCS_DEV fsum2 fsum_pair(fsum2 a, fsum2 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    fsum2 r;
    r.hi = s;
    r.lo = (a.lo + b.lo) + e;
    return r;
}
// Warp-wide sum of (hi, lo) pairs; identical result in every lane.
LRCCS_DEV double warp_fsum(fsum2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o), ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
        float s, e;
        // order the pair so that both lanes of a butterfly compute the same sum
        const bool first = (threadIdx.x & o) == 0;
        two_sum(first ? v.hi : oh, first ? oh : v.hi, s, e);
        v.lo = (first ? v.lo + ol : ol + v.lo) + e;
        v.hi = s;
    }
    return (double)v.hi + (double)v.lo;
}

// Block-wide compensated sums dst[e] = sum_{m < nitem} fetch(e, m) for
// e < nent, written as FP64 (re, im) pairs.  Thread (entry e, slice s) sums
// items s, s + S, s + 2S, ... in that order with RB loads in flight, and the S
// slices are then combined in order: deterministic, and one memory latency per
// RB items instead of one per item.  All threads of the block call it (the
// first 256 do the work); it ends with a barrier.
template <class F>
LRCCS_DEV void block_sum(int nent, int nitem, double *dst, F fetch) {
    constexpr int RB = 16;
    __shared__ float4 s_acc[256];   // (hi, lo) of re and im per thread
    const int nt = blockDim.x < 256 ? (int)blockDim.x : 256;
    const int t = threadIdx.x;
    const bool act = t < nt;   // threads beyond the first 256 only meet the barriers
    const int S = nent >= nt ? 1 : max(1, min(nt / nent, nitem));
    for (int base = 0; base < nent; base += nt) {
        const int e = base + (S == 1 ? t : t % nent), s = S == 1 ? 0 : t / nent;
        fsum2 re = {0.f, 0.f}, im = {0.f, 0.f};
        if (act && e < nent && s < S) {
            for (int m = s; m < nitem; m += S * RB) {
                float2 v[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int mm = m + u * S;
                    v[u] = mm < nitem ? fetch(e, mm) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    fsum_add(re, v[u].x);
                    fsum_add(im, v[u].y);
                }
            }
        }
        if (S == 1) {
            if (act && e < nent) {
                dst[2 * e] = (double)re.hi + (double)re.lo;
                dst[2 * e + 1] = (double)im.hi + (double)im.lo;
            }
            continue;
        }
        if (act) s_acc[t] = make_float4(re.hi, re.lo, im.hi, im.lo);
        __syncthreads();
        if (t < nent) {
            fsum2 R = {0.f, 0.f}, I = {0.f, 0.f};
            for (int ss = 0; ss < S; ++ss) {
                const float4 a = s_acc[ss * nent + t];
                fsum_add(R, a.x);
                R.lo += a.y;
                fsum_add(I, a.z);
                I.lo += a.w;
            }
            dst[2 * t] = (double)R.hi + (double)R.lo;
            dst[2 * t + 1] = (double)I.hi + (double)I.lo;
        }
    }
    __syncthreads();
}

// Sum nblk rows of float2 partials (row length len, row b at part + b * len)
// into dst (FP64 re, im pairs).
LRCCS_DEV void block_reduce_rows(const float2 *part, int nblk, int len, double *dst) {
    block_sum(len, nblk, dst, [=](int e, int b) { return __ldcg(part + (size_t)b * len + e); });
}

// ---------------------------------------------------------------- grid barrier of a cooperative launch

// Barrier number k (1, 2, ...) of this launch: wait until every block has
// arrived k times (plus `skew` arrivals, which only the timeout test sets and
// the grid can never make).  Bounded: gives up after `limit` polls (2^24, about
// a second) and ORs `timeout_bit` into the status word; the kernel then runs on
// to its end.
LRCCS_DEV void grid_sync(unsigned int *bar, unsigned int k, unsigned int *status, unsigned int limit,
                         unsigned int skew, unsigned int timeout_bit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = k * gridDim.x + skew;
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned int v = 0, spins = 0;
        while (true) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (++spins > limit) {
                atomicOr(status, timeout_bit);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

// ---------------------------------------------------------------- asynchronous global -> shared copies
// cp.async keeps many copies in flight per thread without staging through
// registers; cp_async_wait() waits for all of this thread's copies, after
// which a __syncthreads() publishes the tile to the block.

LRCCS_DEV unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// 8-byte copy (one complex64); src must be 8-byte aligned.
LRCCS_DEV void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// 16-byte copy (two complex64); src and dst must be 16-byte aligned.
LRCCS_DEV void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// Stage `count` complex64 values from global `src` into shared `dst`, 16 bytes
// per copy when both are 16-byte aligned and count is even, else 8 bytes.
LRCCS_DEV void stage_row(float2 *dst, const float2 *src, int count, int tid, int nthr) {
    if (((((uintptr_t)src) | smem_u32(dst)) & 15) == 0 && (count & 1) == 0) {
        for (int e = tid; e < count / 2; e += nthr) cp_async16(dst + 2 * e, src + 2 * e);
    } else {
        for (int e = tid; e < count; e += nthr) cp_async8(dst + e, src + e);
    }
}
LRCCS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
LRCCS_DEV void cp_async_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// wait until at most one committed group is still pending (double buffering)
LRCCS_DEV void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---------------------------------------------------------------- tensor copies (TMA)
// A 2D tile of a tensor map (cp.async.bulk.tensor) lands in shared memory and
// completes a transaction count on an mbarrier: one thread arms the barrier
// with the tile bytes and issues the copies, every thread waits on it.  The
// wait is bounded: false when it gave up.

LRCCS_DEV void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
LRCCS_DEV void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// tile at element coordinates (x, y) of the 2D map into dst (16-byte aligned)
LRCCS_DEV void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
LRCCS_DEV bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
    unsigned done = 0;
    for (unsigned it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// ---------------------------------------------------------------- FP32 r x r factorisation

// In place A = L L^H for a Hermitian r x r A (FP32, row-major, r <= RMAX) by
// one warp, lane i holding row i in registers: the lower triangle of A
// receives L, invd[i] = 1 / L[i][i].  Returns false (every lane) if a pivot
// is not positive.
template <int RMAX>
LRCCS_DEV bool warp_chol32(float2 *A, int r, float *invd) {
    const int i = threadIdx.x & 31;
    float2 row[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) row[j] = (i < r && j <= i) ? A[i * r + j] : make_float2(0.f, 0.f);
    float myinv = 1.f;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < RMAX; ++c) {
        if (c < r && ok) {   // uniform across the warp
            const float d = __shfl_sync(0xffffffffu, row[c].x, c);
            ok = d > 0.f;
            const float is = ok ? rsqrtf(d) : 0.f;
            float2 lic = make_float2(0.f, 0.f);
            if (i == c) {
                lic = make_float2(d * is, 0.f);
                myinv = is;
            } else if (i > c && i < r) {
                lic = cscale(row[c], is);
            }
            if (i >= c) row[c] = lic;
#pragma unroll
            for (int j = c + 1; j < RMAX; ++j) {
                if (j < r) {
                    const float ljx = __shfl_sync(0xffffffffu, lic.x, j), ljy = __shfl_sync(0xffffffffu, lic.y, j);
                    if (i >= j && i < r) {   // A[i][j] -= L[i][c] conj(L[j][c])
                        row[j].x -= lic.x * ljx + lic.y * ljy;
                        row[j].y -= lic.y * ljx - lic.x * ljy;
                    }
                }
            }
        }
    }
    __syncwarp();
    if (ok && i < r) {
#pragma unroll
        for (int j = 0; j < RMAX; ++j)
            if (j < r) A[i * r + j] = j <= i ? row[j] : make_float2(0.f, 0.f);
        invd[i] = myinv;
    }
    __syncwarp();
    return ok;
}

// Solve L L^H x = h (L from warp_chol32, lower triangle of the row-major r x r
// FP32 matrix, invd = 1 / diag) by one warp; lane i holds h_i on entry and
// returns x_i (lanes >= r return 0).  Right-looking substitutions.
LRCCS_DEV float2 warp_chol_solve32(const float2 *L, const float *invd, int r, float2 h) {
    const int i = threadIdx.x & 31;
    for (int c = 0; c < r; ++c) {            // L z = h
        const float2 hc = make_float2(__shfl_sync(0xffffffffu, h.x, c), __shfl_sync(0xffffffffu, h.y, c));
        const float2 z = cscale(hc, invd[c]);
        if (i == c) h = z;
        else if (i > c && i < r) h = csub(h, cmul(L[i * r + c], z));
    }
    for (int c = r - 1; c >= 0; --c) {       // L^H x = z
        const float2 hc = make_float2(__shfl_sync(0xffffffffu, h.x, c), __shfl_sync(0xffffffffu, h.y, c));
        const float2 x = cscale(hc, invd[c]);
        if (i == c) h = x;
        else if (i < c) h = csub(h, cmulc(L[c * r + i], x));
    }
    return i < r ? h : make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------- latency-lean FP64 r x r kernels
// On this GPU a dependent FP64 FMA costs ~64 cycles and an FP64 square root or
// division several hundred, so the r x r factorizations below avoid both: a
// reciprocal square root / reciprocal is seeded in FP32 and refined by one
// Newton step in FP64 (relative error ~1e-14), and every step spreads its
// updates over the lanes of a warp (right-looking forms).

LRCCS_DEV double d_rsqrt(double x) {   // 1/sqrt(x), x > 0
    double y = (double)rsqrtf((float)x);
    const double t = x * y * y;
    return y * fma(-0.5, t, 1.5);
}
LRCCS_DEV double d_rcp(double x) {     // 1/x, x != 0
    const double r = (double)__frcp_rn((float)x);
    return fma(r, fma(-x, r, 1.0), r);
}

// In place A = L L^H (A Hermitian, FP64 (re, im) pairs, row-major, r <= 32):
// the lower triangle of A receives L and invd[c] = 1 / L[c][c].  One warp;
// lane i owns row i of the trailing matrix.  Returns false if A is not
// positive definite (same value in every lane).
LRCCS_DEV bool warp_cholesky_rl(double *A, int r, double *invd) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < r; ++c) {
        const double d = A[(c * r + c) * 2];
        if (!(d > 0.0)) return false;
        const double is = d_rsqrt(d);
        // column c below the diagonal: L[i][c] = A[i][c] / sqrt(d)
        double lr = 0.0, li = 0.0;
        if (lane > c && lane < r) {
            lr = A[(lane * r + c) * 2] * is;
            li = A[(lane * r + c) * 2 + 1] * is;
        }
        __syncwarp();
        if (lane == c) {
            A[(c * r + c) * 2] = d * is;
            A[(c * r + c) * 2 + 1] = 0.0;
            invd[c] = is;
        }
        if (lane > c && lane < r) {
            A[(lane * r + c) * 2] = lr;
            A[(lane * r + c) * 2 + 1] = li;
        }
        __syncwarp();
        // trailing update A[i][j] -= L[i][c] conj(L[j][c]) for c < j <= i, the
        // (r-c-1)(r-c)/2 entries spread over the lanes
        const int rt = r - c - 1;
        for (int e = lane; e < rt * (rt + 1) / 2; e += 32) {
            int a, b;
            pair_of(e, rt, a, b);
            const int j = c + 1 + a, i = c + 1 + b;
            const double ar = A[(i * r + c) * 2], ai = A[(i * r + c) * 2 + 1];
            const double br = A[(j * r + c) * 2], bi = A[(j * r + c) * 2 + 1];
            A[(i * r + j) * 2] -= ar * br + ai * bi;
            A[(i * r + j) * 2 + 1] -= ai * br - ar * bi;
        }
        __syncwarp();
    }
    return true;
}

// Solve L L^H x = h with the factor of warp_cholesky_rl; h and x are r (re, im)
// pairs in shared memory (h is consumed).  Right-looking substitutions.
LRCCS_DEV void warp_chol_solve_rl(const double *L, const double *invd, int r, double *h, double *x) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < r; ++c) {            // L z = h  (z in h)
        const double zr = h[2 * c] * invd[c], zi = h[2 * c + 1] * invd[c];
        __syncwarp();
        if (lane == c) {
            h[2 * c] = zr;
            h[2 * c + 1] = zi;
        }
        if (lane > c && lane < r) {          // h[i] -= L[i][c] z
            const double ar = L[(lane * r + c) * 2], ai = L[(lane * r + c) * 2 + 1];
            h[2 * lane] -= ar * zr - ai * zi;
            h[2 * lane + 1] -= ar * zi + ai * zr;
        }
        __syncwarp();
    }
    for (int c = r - 1; c >= 0; --c) {       // L^H x = z
        const double xr = h[2 * c] * invd[c], xi = h[2 * c + 1] * invd[c];
        __syncwarp();
        if (lane == c) {
            x[2 * c] = xr;
            x[2 * c + 1] = xi;
        }
        if (lane < c) {                      // z[i] -= conj(L[c][i]) x_c
            const double ar = L[(c * r + lane) * 2], ai = -L[(c * r + lane) * 2 + 1];
            h[2 * lane] -= ar * xr - ai * xi;
            h[2 * lane + 1] -= ar * xi + ai * xr;
        }
        __syncwarp();
    }
}
