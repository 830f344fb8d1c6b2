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

// ---------------------------------------------------------------- warp FFT
//
// One warp computes one length-N DFT, N = 32 P (P = 1..8), as a Cooley-Tukey
// split N = 32 x P: a P-point DFT inside each lane, a twiddle, then a 32-point
// radix-2 decimation-in-time DFT across the lanes with warp shuffles.
//   input : lane L holds v[m] = x[brev5(L) + 32 m]
//   output: lane L holds v[k2] = X[k2 + P L]
// tw: table of w_N^t = exp(-2 pi i t / N), t in [0, N) (shared memory);
// inverse = true uses conjugate twiddles (unnormalised: the caller scales).

template <int P>
LRCCS_DEV void warp_fft(float2 (&v)[P], const float2 *__restrict__ tw, bool inverse) {
    constexpr int N = 32 * P;
    const int lane = threadIdx.x & 31;
    const int n1 = brev5(lane);
    const float sg = inverse ? -1.f : 1.f;
    // 1) P-point DFT in registers: Y[k2] = sum_m v[m] w_P^{m k2}, w_P = w_N^32
    if (P > 1) {
        float2 y[P];
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) {
            float2 acc = v[0];
#pragma unroll
            for (int m = 1; m < P; ++m) {
                float2 w = tw[(32 * ((m * k2) % P)) % N];
                w.y *= sg;
                cfma(acc, v[m], w);
            }
            y[k2] = acc;
        }
        // 2) twiddle w_N^{n1 k2}
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) {
            float2 w = tw[(n1 * k2) % N];
            w.y *= sg;
            v[k2] = (k2 == 0) ? y[0] : cmul(y[k2], w);
        }
    }
    // 3) 32-point DIT across lanes (bit-reversed input, natural output)
#pragma unroll
    for (int h = 1; h < 32; h <<= 1) {
        const int j = lane & (h - 1);
        float2 w = tw[(j * (N / (2 * h))) % N];
        w.y *= sg;
        const bool top = (lane & h) == 0;
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) {
            float2 u = shfl_xor2(v[k2], h);
            v[k2] = top ? cadd(v[k2], cmul(w, u)) : csub(u, cmul(w, v[k2]));
        }
    }
}

// Run the transforms of a shared-memory tile: element e of transform t lives
// at tile[e * es + t * ts].  Warp w handles transforms w, w + nwarps, ...
// Results are written back in place, in natural order, scaled by `scale`.
template <int P>
LRCCS_DEV void tile_fft(float2 *tile, int es, int ts, int ntrans, const float2 *tw, bool inverse, float scale) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int n1 = brev5(lane);
    for (int t = warp; t < ntrans; t += nw) {
        float2 v[P];
#pragma unroll
        for (int m = 0; m < P; ++m) v[m] = tile[(n1 + 32 * m) * es + t * ts];
        warp_fft<P>(v, tw, inverse);
        __syncwarp();
#pragma unroll
        for (int k2 = 0; k2 < P; ++k2) tile[(k2 + P * lane) * es + t * ts] = cscale(v[k2], scale);
        __syncwarp();
    }
}

// Load the twiddle table of length N into shared memory.
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
__device__ inline void block_jacobi(float2 *A, int n, float2 *V, int ldv, float *s_c, float *s_s, float2 *s_e,
                             int *s_cnt, int max_sweeps) {
    const int n2 = n + (n & 1);
    const int npair = n2 / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *s_cnt = 0;
        __syncthreads();
        for (int rnd = 0; rnd < n2 - 1; ++rnd) {
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                int p, qq;
                if (i == 0) { p = rnd; qq = n2 - 1; }
                else { p = (rnd + i) % (n2 - 1); qq = (rnd - i + n2 - 1) % (n2 - 1); }
                float c = 1.f, s = 0.f;
                float2 e = make_float2(1.f, 0.f);
                if (p < n && qq < n) {
                    const float2 apq = A[p * n + qq];
                    const float b = hypotf(apq.x, apq.y);
                    const float al = A[p * n + p].x, ga = A[qq * n + qq].x;
                    if (b > 1e-30f && b > 1e-7f * sqrtf(fabsf(al) * fabsf(ga))) {
                        e = make_float2(apq.x / b, apq.y / b);
                        const float tau = (ga - al) / (2.f * b);
                        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
                        c = rsqrtf(1.f + t * t);
                        s = t * c;
                        atomicAdd(s_cnt, 1);
                    }
                }
                s_c[i] = c;
                s_s[i] = s;
                s_e[i] = e;
            }
            __syncthreads();
            // rows p, q: A <- G^H A
            for (int task = threadIdx.x; task < npair * n; task += blockDim.x) {
                const int i = task / n, m = task % n;
                if (s_s[i] == 0.f) continue;
                int p, qq;
                if (i == 0) { p = rnd; qq = n2 - 1; }
                else { p = (rnd + i) % (n2 - 1); qq = (rnd - i + n2 - 1) % (n2 - 1); }
                const float c = s_c[i], s = s_s[i];
                const float2 e = s_e[i];
                const float2 ap = A[p * n + m], aq = A[qq * n + m];
                const float2 eaq = cmul(e, aq);
                A[p * n + m] = make_float2(c * ap.x - s * eaq.x, c * ap.y - s * eaq.y);
                A[qq * n + m] = make_float2(s * ap.x + c * eaq.x, s * ap.y + c * eaq.y);
            }
            __syncthreads();
            // columns p, q: A <- A G ; V <- V G
            for (int task = threadIdx.x; task < npair * n; task += blockDim.x) {
                const int i = task / n, m = task % n;
                if (s_s[i] == 0.f) continue;
                int p, qq;
                if (i == 0) { p = rnd; qq = n2 - 1; }
                else { p = (rnd + i) % (n2 - 1); qq = (rnd - i + n2 - 1) % (n2 - 1); }
                const float c = s_c[i], s = s_s[i];
                const float2 eh = cconj(s_e[i]);
                {
                    const float2 ap = A[m * n + p], aq = A[m * n + qq];
                    const float2 e2 = cmul(eh, aq);
                    A[m * n + p] = make_float2(c * ap.x - s * e2.x, c * ap.y - s * e2.y);
                    A[m * n + qq] = make_float2(s * ap.x + c * e2.x, s * ap.y + c * e2.y);
                }
                if (V) {
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
