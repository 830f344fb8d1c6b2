// fft.cuh -- batched length-N DFTs of shared-memory tiles (N = 32 .. 256, a
// multiple of 32), as a two-pass Cooley-Tukey split N = R1 x R2 with both
// factors done as straight-line register DFTs:
//
//   X[k1 + R1 k2] = sum_{j2} w_N^{j2 k1} w_R2^{j2 k2} sum_m x[j2 + R2 m] w_R1^{m k1}
//
// pass 1 (item = transform, j2): DFT_R1 over m, times w_N^{j2 k1}, back to j2 + R2 k1;
// pass 2 (item = transform, k1): DFT_R2 over j2 of the contiguous block k1,
//                                 written to k1 + R1 k2 (natural order).
// The register DFTs are themselves split (8 = 2x4, 12 = 4x3, 16 = 4x4, ...)
// with twiddle constants evaluated at compile time (own constexpr series).
#pragma once

#include "common.cuh"

namespace fft {

constexpr double kPi = 3.141592653589793238462643383279502884;

// sin / cos by their Taylor series after reduction to [-pi, pi] (compile time).
__host__ __device__ constexpr double series_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double series_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
// exp(-2 pi i j / R): real and imaginary parts
__host__ __device__ constexpr double tw_re(int j, int R) {
    const int jj = ((j % R) + R) % R;
    double a = 2.0 * kPi * (double)jj / (double)R;
    if (a > kPi) a -= 2.0 * kPi;
    return series_cos(a);
}
__host__ __device__ constexpr double tw_im(int j, int R) {
    const int jj = ((j % R) + R) % R;
    double a = 2.0 * kPi * (double)jj / (double)R;
    if (a > kPi) a -= 2.0 * kPi;
    return -series_sin(a);
}

// v * w_R^j (conjugate twiddle when INV), with the trivial angles special-cased.
template <int R, int J, bool INV>
LRCCS_DEV float2 twmul(float2 v) {
    constexpr int j = ((J % R) + R) % R;
    if constexpr (j == 0) {
        return v;
    } else if constexpr (4 * j == R) {        // -i (forward) / +i (inverse)
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (2 * j == R) {        // -1
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * j == 3 * R) {    // +i (forward) / -i (inverse)
        return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    } else {
        constexpr float c = (float)tw_re(j, R);
        constexpr float s = INV ? (float)-tw_im(j, R) : (float)tw_im(j, R);
        return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
    }
}

// In-register DFT of length R, natural order in and out, unnormalised.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<1, INV> {
    static LRCCS_DEV void run(float2 *) {}
};

template <bool INV>
struct Dft<2, INV> {
    static LRCCS_DEV void run(float2 *v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<3, INV> {
    static LRCCS_DEV void run(float2 *v) {
        constexpr float c1 = -0.5f;
        constexpr float s1 = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
        const float2 a = v[0], b = v[1], c = v[2];
        const float2 t = cadd(b, c), d = csub(b, c);
        v[0] = cadd(a, t);
        const float2 m = make_float2(a.x + c1 * t.x, a.y + c1 * t.y);
        const float2 j = make_float2(-s1 * d.y, s1 * d.x);   // i * s1 * d
        v[1] = cadd(m, j);
        v[2] = csub(m, j);
    }
};

template <bool INV>
struct Dft<4, INV> {
    static LRCCS_DEV void run(float2 *v) {
        const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        const float2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
        // forward: X1 = a1 - i b1, X3 = a1 + i b1
        const float2 ib1 = INV ? make_float2(-b1.y, b1.x) : make_float2(b1.y, -b1.x);
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, ib1);
        v[3] = csub(a1, ib1);
    }
};

template <bool INV>
struct Dft<5, INV> {
    static LRCCS_DEV void run(float2 *v) {
        constexpr float c1 = (float)tw_re(1, 5), c2 = (float)tw_re(2, 5);
        constexpr float s1 = INV ? (float)-tw_im(1, 5) : (float)tw_im(1, 5);
        constexpr float s2 = INV ? (float)-tw_im(2, 5) : (float)tw_im(2, 5);
        const float2 x0 = v[0];
        const float2 p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
        const float2 p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
        v[0] = make_float2(x0.x + p1.x + p2.x, x0.y + p1.y + p2.y);
        const float2 r1 = make_float2(x0.x + c1 * p1.x + c2 * p2.x, x0.y + c1 * p1.y + c2 * p2.y);
        const float2 r2 = make_float2(x0.x + c2 * p1.x + c1 * p2.x, x0.y + c2 * p1.y + c1 * p2.y);
        // i (s1 m1 + s2 m2) and i (s2 m1 - s1 m2)
        const float2 q1 = make_float2(-(s1 * m1.y + s2 * m2.y), s1 * m1.x + s2 * m2.x);
        const float2 q2 = make_float2(-(s2 * m1.y - s1 * m2.y), s2 * m1.x - s1 * m2.x);
        v[1] = cadd(r1, q1);
        v[4] = csub(r1, q1);
        v[2] = cadd(r2, q2);
        v[3] = csub(r2, q2);
    }
};

template <bool INV>
struct Dft<7, INV> {
    // outputs k and 7 - k from the sums p_a = x_a + x_{7-a} and differences m_a = x_a - x_{7-a}
    template <int K>
    static LRCCS_DEV void pair(const float2 x0, const float2 *p, const float2 *m, float2 *v) {
        constexpr float c1 = (float)tw_re(K * 1, 7), c2 = (float)tw_re(K * 2, 7), c3 = (float)tw_re(K * 3, 7);
        constexpr float s1 = INV ? (float)-tw_im(K * 1, 7) : (float)tw_im(K * 1, 7);
        constexpr float s2 = INV ? (float)-tw_im(K * 2, 7) : (float)tw_im(K * 2, 7);
        constexpr float s3 = INV ? (float)-tw_im(K * 3, 7) : (float)tw_im(K * 3, 7);
        const float2 rr = make_float2(x0.x + c1 * p[0].x + c2 * p[1].x + c3 * p[2].x,
                                      x0.y + c1 * p[0].y + c2 * p[1].y + c3 * p[2].y);
        // i (s1 m0 + s2 m1 + s3 m2)
        const float2 qq = make_float2(-(s1 * m[0].y + s2 * m[1].y + s3 * m[2].y),
                                      s1 * m[0].x + s2 * m[1].x + s3 * m[2].x);
        v[K] = cadd(rr, qq);
        v[7 - K] = csub(rr, qq);
    }
    static LRCCS_DEV void run(float2 *v) {
        const float2 x0 = v[0];
        float2 p[3], m[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p[a] = cadd(v[1 + a], v[6 - a]);
            m[a] = csub(v[1 + a], v[6 - a]);
        }
        v[0] = make_float2(x0.x + p[0].x + p[1].x + p[2].x, x0.y + p[0].y + p[1].y + p[2].y);
        pair<1>(x0, p, m, v);
        pair<2>(x0, p, m, v);
        pair<3>(x0, p, m, v);
    }
};

// Composite R = P x Q: x[Q n1 + n2] -> X[k1 + P k2].
template <int P, int Q, bool INV>
struct DftSplit {
    static LRCCS_DEV void run(float2 *v) {
        constexpr int R = P * Q;
        float2 a[R];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            float2 t[P];
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) t[n1] = v[Q * n1 + n2];
            Dft<P, INV>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) a[n2 * P + k1] = t[k1];
        }
        twiddle_all<0>(a);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            float2 t[Q];
#pragma unroll
            for (int n2 = 0; n2 < Q; ++n2) t[n2] = a[n2 * P + k1];
            Dft<Q, INV>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
        }
    }
    // a[n2 P + k1] *= w_R^{n2 k1}
    template <int E>
    static LRCCS_DEV void twiddle_all(float2 *a) {
        if constexpr (E < P * Q) {
            constexpr int n2 = E / P, k1 = E % P;
            a[E] = twmul<P * Q, n2 * k1, INV>(a[E]);
            twiddle_all<E + 1>(a);
        }
    }
};

template <bool INV> struct Dft<6, INV> : DftSplit<2, 3, INV> {};
template <bool INV> struct Dft<8, INV> : DftSplit<2, 4, INV> {};
template <bool INV> struct Dft<10, INV> : DftSplit<2, 5, INV> {};
template <bool INV> struct Dft<12, INV> : DftSplit<4, 3, INV> {};
template <bool INV> struct Dft<14, INV> : DftSplit<2, 7, INV> {};
template <bool INV> struct Dft<16, INV> : DftSplit<4, 4, INV> {};

// Factorisation N = R1 x R2 used for each supported length.
template <int N> struct Plan;
template <> struct Plan<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct Plan<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Plan<96> { static constexpr int R1 = 12, R2 = 8; };
template <> struct Plan<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct Plan<160> { static constexpr int R1 = 10, R2 = 16; };
template <> struct Plan<192> { static constexpr int R1 = 12, R2 = 16; };
template <> struct Plan<224> { static constexpr int R1 = 14, R2 = 16; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16; };

// Transform `ntrans` length-N sequences of a shared-memory tile in place:
// element e of transform t at tile[e * es + t].  tw: w_N^t, t < N (shared).
// Every thread of the block must call it (it synchronises).
template <int N, bool INV>
LRCCS_DEV void tile_dft(float2 *tile, int es, int ntrans, const float2 *__restrict__ tw, float scale) {
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // pass 1: DFT_R1 over m of x[j2 + R2 m], times w_N^{j2 k1}.  Requires
    // ntrans <= blockDim.x: thread -> transform t = tid % ntrans (fixed) and
    // j2 = tid / ntrans, stepping by the number of thread groups.
    const int ngrp = nthr / ntrans;
    const int t = tid % ntrans, g0 = tid / ntrans;
    for (int j2 = (g0 < ngrp ? g0 : R2); j2 < R2; j2 += ngrp) {
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = tile[(j2 + R2 * m) * es + t];
        Dft<R1, INV>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 w = tw[j2 * k1];
            if (INV) w.y = -w.y;
            tile[(j2 + R2 * k1) * es + t] = (k1 == 0) ? v[0] : cmul(v[k1], w);
        }
    }
    __syncthreads();
    // pass 2: DFT_R2 of block k1, stored to k1 + R1 k2 (in chunks of transforms)
    const int tc = max(1, nthr / R1);
    for (int t0 = 0; t0 < ntrans; t0 += tc) {
        const int tn = min(tc, ntrans - t0);
        const int it = tid;
        const bool act = it < tn * R1;
        const int t = t0 + (act ? it % tn : 0), k1 = act ? it / tn : 0;
        float2 v[R2];
        if (act) {
#pragma unroll
            for (int j2 = 0; j2 < R2; ++j2) v[j2] = tile[(j2 + R2 * k1) * es + t];
            Dft<R2, INV>::run(v);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) tile[(k1 + R1 * k2) * es + t] = cscale(v[k2], scale);
        }
        __syncthreads();
    }
}

// The same transform with the tile's first read and last write replaced:
// pass 1 reads element `row` of transform t as load(row, t) (e.g. the tile
// times a coil map), and pass 2 hands each output (transform t, natural row,
// unscaled value) to epi(t, row, v) instead of storing it into the tile (e.g.
// a store to global memory, or an accumulation in registers).  Pass 2 only
// reads the tile, so it has no barriers; a caller that reuses the tile after
// it must synchronise.  Every thread of the block must call it.
template <int N, bool INV, class LOAD, class EPI>
LRCCS_DEV void tile_dft_io(float2 *tile, int es, int ntrans, const float2 *__restrict__ tw, LOAD load, EPI epi) {
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ngrp = nthr / ntrans;
    const int t = tid % ntrans, g0 = tid / ntrans;
    for (int j2 = (g0 < ngrp ? g0 : R2); j2 < R2; j2 += ngrp) {
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = load(j2 + R2 * m, t);
        Dft<R1, INV>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 w = tw[j2 * k1];
            if (INV) w.y = -w.y;
            tile[(j2 + R2 * k1) * es + t] = (k1 == 0) ? v[0] : cmul(v[k1], w);
        }
    }
    __syncthreads();
    const int tc = max(1, nthr / R1);
    for (int t0 = 0; t0 < ntrans; t0 += tc) {
        const int tn = min(tc, ntrans - t0);
        if (tid < tn * R1) {
            const int tt = t0 + tid % tn, k1 = tid / tn;
            float2 v[R2];
#pragma unroll
            for (int j2 = 0; j2 < R2; ++j2) v[j2] = tile[(j2 + R2 * k1) * es + tt];
            Dft<R2, INV>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) epi(tt, k1 + R1 * k2, v[k2]);
        }
    }
}

// Pass 1 as in tile_dft (in place), then pass 2 hands every output to
// epi(ch, k2, t, row, v) with the chunk ch < NCH and k2 < R2 as compile-time
// constants after unrolling, so a caller can keep per-thread accumulators in
// registers: a thread sees the same (t, row) for a given (ch, k2) on every
// call with the same ntrans.  Requires ceil(ntrans / (blockDim.x / R1)) <= NCH.
// Pass 2 only reads the tile (no barriers after pass 1).
template <int N, bool INV, int NCH, class EPI>
LRCCS_DEV void tile_dft_acc(float2 *tile, int es, int ntrans, const float2 *__restrict__ tw, EPI epi) {
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ngrp = nthr / ntrans;
    const int t = tid % ntrans, g0 = tid / ntrans;
    for (int j2 = (g0 < ngrp ? g0 : R2); j2 < R2; j2 += ngrp) {
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = tile[(j2 + R2 * m) * es + t];
        Dft<R1, INV>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 w = tw[j2 * k1];
            if (INV) w.y = -w.y;
            tile[(j2 + R2 * k1) * es + t] = (k1 == 0) ? v[0] : cmul(v[k1], w);
        }
    }
    __syncthreads();
    const int tc = max(1, nthr / R1);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const int t0 = ch * tc;
        const int tn = min(tc, ntrans - t0);
        if (t0 < ntrans && tid < tn * R1) {
            const int tt = t0 + tid % tn, k1 = tid / tn;
            float2 v[R2];
#pragma unroll
            for (int j2 = 0; j2 < R2; ++j2) v[j2] = tile[(j2 + R2 * k1) * es + tt];
            Dft<R2, INV>::run(v);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) epi(ch, k2, tt, k1 + R1 * k2, v[k2]);
        }
    }
}

// The (chunk, k2) -> (t, row) map of tile_dft_acc's pass 2 for this thread:
// f(ch, k2, t, row) for every output it owns (e.g. to write its accumulators).
template <int N, int NCH, class F>
LRCCS_DEV void tile_dft_acc_slots(int ntrans, F f) {
    constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
    const int tid = threadIdx.x, tc = max(1, (int)blockDim.x / R1);
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const int t0 = ch * tc;
        const int tn = min(tc, ntrans - t0);
        if (t0 < ntrans && tid < tn * R1) {
            const int tt = t0 + tid % tn, k1 = tid / tn;
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) f(ch, k2, tt, k1 + R1 * k2);
        }
    }
}

}  // namespace fft
