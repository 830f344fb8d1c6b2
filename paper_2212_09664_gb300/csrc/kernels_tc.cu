// kernels_tc.cu -- the precision forms of the forward column transform on the
// 5th-generation tensor cores (tcgen05, sm_103a): the DFT along ky over the
// sampled phase-encode rows as a dense GEMM (Sec. II-A's A_k U with F written
// as a matrix), instead of the FP32 FFT of k_fwd_cols.
//
// Per coil j the sampled rows of T_j = F_y (d_j o U) are
//     T_j[ky_s, (x, l)] = sum_y F[ky_s, y] (d_j o U)[y, (x, l)],
// a complex (n_used x ny) x (ny x nx r) product, done as one real GEMM
//     C (2 n_used x N) = A (2 n_used x 2 ny) B (2 ny x N),   N = nx r,
// with rows m = 2 s + c (c = 0: real part of output row s, 1: imaginary) and
// columns k = 2 y + c' (c' = 0: real, 1: imaginary part of the input), so that
// A[(s,0), (y,0)] = Re F, A[(s,0), (y,1)] = -Im F, A[(s,1), (y,0)] = Im F,
// A[(s,1), (y,1)] = Re F.  Two precision forms, both accumulating in FP32 in
// tensor memory:
//   BF16X3 : A = A_hi + A_lo and B = B_hi + B_lo (bf16 each); C = A_hi B_hi +
//            A_hi B_lo + A_lo B_hi (three MMA passes over K; the dropped
//            A_lo B_lo term is ~2^-16 relative);
//   FP16S  : one pass in FP16; every CTA scales its B tile by a power of two
//            chosen from the tile's largest entry (per-tile scaling) and
//            unscales the accumulator.
// A depends only on the sampled rows: k_dft_a builds it once per data load in
// the operand layout the MMA reads (bf16 hi / lo, or fp16).  B is formed by
// the CTA's threads from U and d_j (coil multiply, split, convert) straight
// into shared memory.
//
// Tiles: M = 128 output rows (64 sampled rows), N = 128 columns, K chunks of
// 64 (32 y values); one CTA of 256 threads per (M tile, N tile, coil).  Each
// chunk: all threads write the A and B tiles to shared memory in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix),
// one thread issues the tcgen05.mma instructions (M 128, N 128, K 16) and
// commits them to an mbarrier, which every thread waits on (bounded) before the
// next chunk overwrites the tiles.  The epilogue reads the accumulator from
// tensor memory (tcgen05.ld), pairs real and imaginary rows through a warp
// shuffle and writes T_j[ky_s] as complex64.
#include <math.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

#define TC_M 128
#define TC_N 128
#define TC_KC 64                       // K per chunk (32 y values, re and im)
#define TC_TILE (TC_M * TC_KC)         // elements of one operand tile (128 x 64)
#define TC_THREADS 256
// no-swizzle K-major layout: core matrix (8 rows x 8 elements, 128 bytes)
// (rg, kb) at (rg * (TC_KC / 8) + kb) * 128 bytes; adjacent core matrices
// along K are 128 bytes apart, along M/N 1024 bytes apart
#define TC_KSTRIDE 128u
#define TC_MSTRIDE 1024u

LRCCS_DEV uint32_t tc_off(int row, int k) {   // byte offset of element (row, k) in a 128 x 64 tile
    return (uint32_t)((((row >> 3) * (TC_KC / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

LRCCS_DEV uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((TC_KSTRIDE >> 4) & 0x3FFF) << 16;   // leading dimension (K) byte offset
    d |= (uint64_t)((TC_MSTRIDE >> 4) & 0x3FFF) << 32;   // stride dimension (M/N) byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version of tcgen05
    return d;                                            // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: FP32 accumulate, A and B both BF16 (bf16 =
// 1) or both FP16 (bf16 = 0), K-major A and B, N = 128, M = 128.
LRCCS_DEV uint32_t tc_idesc(int bf16) {
    const uint32_t ab = bf16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

LRCCS_DEV void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
LRCCS_DEV bool tc_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// ---------------------------------------------------------------- A operand

// A for the sampled rows usedrows[0 .. n_used) in tiles of 128 x 64 (tile
// (bm, kc) at (bm * KC + kc) * TC_TILE elements), F[ky, y] = exp(-2 pi i ky y /
// ny) / sqrt(ny) in FP64, rows past 2 n_used zero.  mode 1: bf16 hi at A0, lo
// at A1; mode 2: fp16 at A0.
__global__ void k_dft_a(const int32_t *__restrict__ usedrows, int n_used, int ny, int mtiles, int mode,
                        uint16_t *__restrict__ A0, uint16_t *__restrict__ A1) {
    const int K2 = 2 * ny, KC = K2 / TC_KC;
    const size_t total = (size_t)mtiles * TC_M * K2;
    const double sc = 1.0 / sqrt((double)ny);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / K2), k = (int)(e % K2);
        const int s = m >> 1, c = m & 1, y = k >> 1, cp = k & 1;
        double v = 0.0;
        if (s < n_used) {
            const int ky = usedrows[s];
            const long long t = ((long long)ky * y) % ny;
            double sn, cs;
            sincospi(-2.0 * (double)t / (double)ny, &sn, &cs);   // F = (cs + i sn) / sqrt(ny)
            const double fr = cs * sc, fi = sn * sc;
            v = c == 0 ? (cp == 0 ? fr : -fi) : (cp == 0 ? fi : fr);
        }
        const int bm = m / TC_M, r = m % TC_M, kc = k / TC_KC, kk = k % TC_KC;
        const size_t o = ((size_t)bm * KC + kc) * TC_TILE + (tc_off(r, kk) >> 1);
        if (mode == 1) {
            const __nv_bfloat16 hi = __double2bfloat16(v);
            const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
            A0[o] = __bfloat16_as_ushort(hi);
            A1[o] = __bfloat16_as_ushort(lo);
        } else {
            A0[o] = __half_as_ushort(__double2half(v));
        }
    }
}

// ---------------------------------------------------------------- FP16S scales

// Per N tile (128 columns (x, l) of U): the power of two that puts the tile's
// largest possible coil product near 2^14 (FP16 holds up to 65504):
// max |d_j o U| <= max |d| max_tile |U|, with max |d| over every coil and pixel
// taken at data load (dmax).
__global__ void __launch_bounds__(TC_N) k_tile_scale(const float2 *__restrict__ U, int ny, int N, const float *dmax,
                                                     float *__restrict__ tscale) {
    __shared__ float s_m[TC_N / 32];
    const int ng = blockIdx.x * TC_N + threadIdx.x;
    float mx = 0.f;
    if (ng < N)
        for (int y = 0; y < ny; ++y) {
            const float2 u = U[(size_t)y * N + ng];
            mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
        }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < TC_N / 32; ++w) m = fmaxf(m, s_m[w]);
        m *= *dmax;
        tscale[blockIdx.x] = m > 0.f ? ldexpf(1.f, 14 - (int)ceilf(log2f(m))) : 1.f;
    }
}

// dmax = 2 max(|Re|, |Im|) >= max |d| over the coil maps (once per data load;
// *dmax zeroed first).  Non-negative floats order like their bit patterns, so
// the blocks combine with an integer atomicMax.
__global__ void k_map_max(const float2 *__restrict__ smaps, size_t count, float *dmax) {
    __shared__ float s_m[8];
    float mx = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fmaxf(fabsf(smaps[e].x), fabsf(smaps[e].y)));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_m[w]);
        atomicMax((int *)dmax, __float_as_int(2.f * m));   // |d| <= |Re| + |Im|
    }
}

// ---------------------------------------------------------------- the GEMM

template <int MODE, int NSTAGE>   // MODE 1 = BF16X3, 2 = FP16S; NSTAGE shared-memory stages (1 or 2)
__global__ void __launch_bounds__(TC_THREADS) k_fwd_gemm(const float2 *__restrict__ U,
                                                         const float2 *__restrict__ smaps,
                                                         const uint16_t *__restrict__ A0,
                                                         const uint16_t *__restrict__ A1,
                                                         const int32_t *__restrict__ usedrows,
                                                         const float *__restrict__ tscale, float2 *__restrict__ T,
                                                         int ny, int nx, int r, int n_used, unsigned int *status) {
    constexpr int NT = MODE == 1 ? 4 : 2;   // operand tiles: A_hi, A_lo, B_hi, B_lo | A, B
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    // NSTAGE stages of NT tiles: with two, chunk kc is produced into stage
    // kc & 1 while the MMAs of chunk kc - 1 read the other stage
    constexpr int STAGE = NT * TC_TILE * 2;   // bytes per stage
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x;
    const int bm = blockIdx.x, n0 = blockIdx.y * TC_N, j = blockIdx.z;
    const int N = nx * r, K2 = 2 * ny, KC = K2 / TC_KC;
    const size_t n = (size_t)ny * nx;
    // this thread's column of B: n = t % 128, and core-matrix columns kb =
    // t / 128, t / 128 + 2, ... of each chunk (4 y values, 8 k, one 16-byte row each)
    const int bn = t & (TC_N - 1), kb0 = t >> 7;
    const int ng = n0 + bn;
    const bool col_ok = ng < N;
    const int x = col_ok ? ng / r : 0;
    const float2 *Ucol = U + (col_ok ? ng : 0);           // U[y nx r + ng]
    const float2 *Scol = smaps + (size_t)j * n + x;       // d_j[y nx + x]
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(&mbar[0]);
    const uint32_t mb1 = (uint32_t)__cvta_generic_to_shared(&mbar[1]);
    // FP16S: the power-of-two scale of this N tile's B (k_tile_scale)
    float bscale = 1.f, binv = 1.f;
    if (MODE == 2) {
        bscale = tscale[blockIdx.y];
        binv = 1.f / bscale;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(
            (uint32_t)__cvta_generic_to_shared(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok = true;
    for (int kc = 0; kc < KC; ++kc) {
        // the stage was last read by the MMAs of chunk kc - NSTAGE (barrier use
        // kc / NSTAGE - 1 of that stage's mbarrier)
        const int st = NSTAGE == 2 ? (kc & 1) : 0;
        const uint32_t mbs = st ? mb1 : mb0;
        const int use = NSTAGE == 2 ? (kc >> 1) : kc;
        if (kc >= NSTAGE && !tc_wait(mbs, (uint32_t)((use - 1) & 1))) ok = false;
        if (!__syncthreads_and(ok)) break;
        uint8_t *sA0 = tc_smem + st * STAGE, *sA1 = sA0 + TC_TILE * 2;
        uint8_t *sB0 = sA0 + (NT / 2) * TC_TILE * 2, *sB1 = sB0 + TC_TILE * 2;
        // A tiles: contiguous 16 KB copies
        {
            const uint4 *g0 = (const uint4 *)(A0 + ((size_t)bm * KC + kc) * TC_TILE);
            for (int e = t; e < TC_TILE * 2 / 16; e += TC_THREADS) ((uint4 *)sA0)[e] = g0[e];
            if (MODE == 1) {
                const uint4 *g1 = (const uint4 *)(A1 + ((size_t)bm * KC + kc) * TC_TILE);
                for (int e = t; e < TC_TILE * 2 / 16; e += TC_THREADS) ((uint4 *)sA1)[e] = g1[e];
            }
        }
        // B tile: for each of this thread's core-matrix columns kb, the coil
        // products of its column for 4 consecutive y (8 k: re, im), split or
        // scaled and converted, stored as one 16-byte row of the core matrix
        for (int kb = kb0; kb < TC_KC / 8; kb += TC_THREADS / TC_N) {
            const int y0 = kc * (TC_KC / 2) + 4 * kb;
            uint32_t w0[4], w1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 p = make_float2(0.f, 0.f);
                if (col_ok) p = cmul(__ldg(Scol + (size_t)(y0 + i) * nx), __ldg(Ucol + (size_t)(y0 + i) * nx * r));
                if (MODE == 1) {
                    const __nv_bfloat16 hr = __float2bfloat16(p.x), hi = __float2bfloat16(p.y);
                    const __nv_bfloat16 lr = __float2bfloat16(p.x - __bfloat162float(hr));
                    const __nv_bfloat16 li = __float2bfloat16(p.y - __bfloat162float(hi));
                    w0[i] = (uint32_t)__bfloat16_as_ushort(hr) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
                    w1[i] = (uint32_t)__bfloat16_as_ushort(lr) | ((uint32_t)__bfloat16_as_ushort(li) << 16);
                } else {
                    w0[i] = (uint32_t)__half_as_ushort(__float2half(p.x * bscale)) |
                            ((uint32_t)__half_as_ushort(__float2half(p.y * bscale)) << 16);
                }
            }
            const uint32_t o = tc_off(bn, 8 * kb);
            *(uint4 *)(sB0 + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
            if (MODE == 1) *(uint4 *)(sB1 + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t idesc = tc_idesc(MODE == 1);
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA0), a1 = (uint32_t)__cvta_generic_to_shared(sA1);
            const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(sB0), b1 = (uint32_t)__cvta_generic_to_shared(sB1);
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
                const uint32_t ko = ks * 2 * 128;   // two K core matrices per MMA
                tc_mma(tmem, tc_desc(a0 + ko), tc_desc(b0 + ko), idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                if (MODE == 1) {
                    tc_mma(tmem, tc_desc(a0 + ko), tc_desc(b1 + ko), idesc, 1u);
                    tc_mma(tmem, tc_desc(a1 + ko), tc_desc(b0 + ko), idesc, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbs));
        }
    }
    // the last commit covers every earlier MMA of this thread
    {
        const int st = NSTAGE == 2 ? ((KC - 1) & 1) : 0, use = NSTAGE == 2 ? ((KC - 1) >> 1) : (KC - 1);
        if (ok && !tc_wait(st ? mb1 : mb0, (uint32_t)(use & 1))) ok = false;
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        // epilogue: warp w reads rows 32 (w % 4) .. + 31 (TMEM lanes), columns
        // 64 (w / 4) .. + 63; the even lane of a pair holds the real part of
        // output row s, the odd lane its imaginary part
        const int w = t >> 5, lane = t & 31;
        const int row = 32 * (w & 3) + lane, cb = 64 * (w >> 2);
        const int s = (bm * TC_M + row) >> 1;
        const bool odd = lane & 1;
        const int ky = s < n_used ? usedrows[s] : -1;
        float2 *Trow = T + ((size_t)j * ny + (ky < 0 ? 0 : ky)) * N;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(cb + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float mine = __uint_as_float(v[i]) * binv;
                const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                // even lanes write the first 8 columns of the 16, odd lanes the last 8
                const int col = n0 + cb + c0 + i;
                if (ky >= 0 && col < N && ((i < 8) != odd))
                    Trow[col] = odd ? make_float2(other, mine) : make_float2(mine, other);
            }
        }
    } else if (t == 0) {
        atomicOr(status, (unsigned)ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
}

// ---------------------------------------------------------------- launchers

int tc_mtiles(int n_used) { return (2 * n_used + TC_M - 1) / TC_M; }
size_t tc_a_elems(int ny) { return (size_t)((2 * ny + TC_M - 1) / TC_M) * TC_M * 2 * ny; }   // per array, worst case

cudaError_t launch_dft_a(lrccs_ctx *c) {
    const int mode = c->dims.precision == LRCCS_PREC_BF16X3_GEMM ? 1 : 2;
    prof_begin(c, KID_TC_A);
    k_dft_a<<<4 * 152, 256, 0, c->stream>>>(c->d_usedrows, c->n_used, c->ny, tc_mtiles(c->n_used), mode, c->d_tcA0,
                                            c->d_tcA1);
    prof_end(c, KID_TC_A);
    if (mode == 2) {
        prof_begin(c, KID_TC_A);
        cudaMemsetAsync(c->d_tcscale, 0, sizeof(float), c->stream);
        k_map_max<<<152, 256, 0, c->stream>>>(c->d_smaps, (size_t)c->nc * c->n, c->d_tcscale);
        prof_end(c, KID_TC_A);
    }
    return cudaGetLastError();
}

cudaError_t launch_fwd_gemm(lrccs_ctx *c) {
    const int N = c->nx * c->r;
    dim3 grid(tc_mtiles(c->n_used), (N + TC_N - 1) / TC_N, c->nc);
    cudaError_t e;
    if (c->dims.precision == LRCCS_PREC_FP16S_GEMM) {
        prof_begin(c, KID_TC_SCALE);
        k_tile_scale<<<(N + TC_N - 1) / TC_N, TC_N, 0, c->stream>>>(c->d_U, c->ny, N, c->d_tcscale,
                                                                    c->d_tcscale + 1);
        prof_end(c, KID_TC_SCALE);
    }
    prof_begin(c, KID_TC_GEMM);
    if (c->dims.precision == LRCCS_PREC_BF16X3_GEMM)
        // one stage of 4 tiles (64 KB): three CTAs per SM overlap one another's
        // operand production and MMAs (two stages, 128 KB, measured slower)
        k_fwd_gemm<1, 1><<<grid, TC_THREADS, 4 * TC_TILE * 2, c->stream>>>(c->d_U, c->d_smaps, c->d_tcA0, c->d_tcA1,
                                                                         c->d_usedrows, c->d_tcscale + 1, c->d_T, c->ny, c->nx,
                                                                         c->r, c->n_used, c->d_status);
    else
        // two stages of 2 tiles (64 KB): at most 3 CTAs per SM, so their
        // 128-column tensor-memory allocations always fit in 512
        k_fwd_gemm<2, 2><<<grid, TC_THREADS, 4 * TC_TILE * 2, c->stream>>>(c->d_U, c->d_smaps, c->d_tcA0, c->d_tcA1,
                                                                         c->d_usedrows, c->d_tcscale + 1, c->d_T, c->ny, c->nx,
                                                                         c->r, c->n_used, c->d_status);
    prof_end(c, KID_TC_GEMM);
    e = cudaGetLastError();
    return e;
}

cudaError_t configure_kernels_tc(int max_smem) {
    cudaError_t e = allow_smem(k_fwd_gemm<1, 1>, max_smem);
    if (e == cudaSuccess) e = allow_smem(k_fwd_gemm<2, 2>, max_smem);
    return e;
}
