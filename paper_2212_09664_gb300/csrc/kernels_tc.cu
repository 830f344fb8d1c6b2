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
//   FP16S  : one pass in FP16; B is scaled per N tile by a power of two
//            chosen from the tile's largest entry (per-tile scaling) and the
//            accumulator is unscaled.
// A depends only on the sampled rows: k_dft_a builds it once per data load in
// the operand layout the MMA reads (bf16 hi / lo, or fp16).  B (d_j o U) is
// built once per transform by k_b_operand in the same tiled layout (coil
// multiply, split or scale, convert), so that the GEMM only moves tiles and
// issues MMAs.
//
// Tiles: M = 128 output rows (64 sampled rows), N = 128 columns, K chunks of
// 32 (16 y values); one CTA of 256 threads per (N tile, coil) covers every M
// tile (up to four accumulators of 128 columns in tensor memory), so each B
// tile is read once.  Thread 0 (producer) streams the chunks' A and B tiles
// into two shared-memory stages with bulk asynchronous copies
// (cp.async.bulk, completing on the stage's "full" mbarrier); thread 32 (MMA
// issuer) waits for a stage, issues tcgen05.mma (M 128, N 128, K 16) for every
// M tile and commits to the stage's "empty" mbarrier, which the producer
// waits on before it refills the stage; the last commit arms a "done"
// mbarrier for the epilogue.  Every wait is bounded.  The epilogue reads the
// accumulators from tensor memory (tcgen05.ld), pairs real and imaginary rows
// through a warp shuffle and writes T_j[ky_s] as complex64.
#include <math.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

#define TC_M 128
#define TC_N 128
#define TC_KC 32                       // K per chunk (16 y values, re and im)
#define TC_TILE (TC_M * TC_KC)         // elements of one operand tile (128 x 32)
#define TC_TILE_BYTES (TC_TILE * 2)
#define TC_THREADS 256
#define TC_MT_MAX 4                    // M tiles per CTA (2 ny / 128 for ny <= 256)
// no-swizzle K-major layout: core matrix (8 rows x 8 elements, 128 bytes)
// (rg, kb) at (rg * (TC_KC / 8) + kb) * 128 bytes; adjacent core matrices
// along K are 128 bytes apart, along M/N 512 bytes apart
#define TC_KSTRIDE 128u
#define TC_MSTRIDE ((TC_KC / 8) * 128u)

LRCCS_DEV uint32_t tc_off(int row, int k) {   // byte offset of element (row, k) in a 128 x 32 tile
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
    for (int it = 0; it < (1 << 22) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// ---------------------------------------------------------------- A operand

// A for the sampled rows usedrows[0 .. n_used) in tiles of 128 x 32 (tile
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

// Per N tile (128 columns (x, l) of U) the largest |Re| or |Im| of U, over
// row blocks of TS_ROWS rows in parallel: block (nb, yb) reduces its rows and
// columns and combines into umax[nb] by an integer atomicMax (non-negative
// floats order like their bit patterns; umax zeroed first).
#define TS_ROWS 16
__global__ void __launch_bounds__(TC_N) k_tile_max(const float2 *__restrict__ U, int ny, int N,
                                                   float *__restrict__ umax) {
    __shared__ float s_m[TC_N / 32];
    const int ng = blockIdx.x * TC_N + threadIdx.x, y0 = blockIdx.y * TS_ROWS;
    float mx = 0.f;
    if (ng < N)
        for (int y = y0; y < min(ny, y0 + TS_ROWS); ++y) {
            const float2 u = U[(size_t)y * N + ng];
            mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
        }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < TC_N / 32; ++w) m = fmaxf(m, s_m[w]);
        atomicMax((int *)(umax + blockIdx.x), __float_as_int(m));
    }
}

// The power of two that puts an N tile's largest possible coil product near
// 2^14 (FP16 holds up to 65504): max |d_j o U| <= max |d| max_tile |U|, with
// max |d| over every coil and pixel taken at data load (dmax).
LRCCS_DEV float tile_scale(float umax, float dmax) {
    const float m = umax * dmax;
    return m > 0.f ? ldexpf(1.f, 14 - (int)ceilf(log2f(m))) : 1.f;
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

// ---------------------------------------------------------------- B operand

// B_j = d_j o U (2 ny x N real, k = 2 y + c') as tiles (coil j, N tile nb,
// K chunk kc) of 128 x 32 at ((j NB + nb) KC + kc) TC_TILE elements: thread =
// (column bn of the tile, core-matrix columns kb, kb + 2: 4 y values each),
// one 16-byte core-matrix row per kb, split (BF16X3) or scaled by the N
// tile's power of two (FP16S) and converted.  Columns past N are zero.
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_b_operand(const float2 *__restrict__ U,
                                                          const float2 *__restrict__ smaps,
                                                          const float *__restrict__ tmax, uint16_t *__restrict__ B0,
                                                          uint16_t *__restrict__ B1, int ny, int nx, int r) {
    const int nb = blockIdx.x, kc = blockIdx.y, j = blockIdx.z, NB = gridDim.x, KC = gridDim.y;
    const int N = nx * r, t = threadIdx.x, bn = t & (TC_N - 1);
    const int ng = nb * TC_N + bn;
    const bool col_ok = ng < N;
    const int x = col_ok ? ng / r : 0;
    const float2 *Ucol = U + (col_ok ? ng : 0);
    const float2 *Scol = smaps + (size_t)j * ny * nx + x;
    const float bscale = MODE == 2 ? tile_scale(tmax[nb], tmax[-1]) : 1.f;   // tmax[-1] = max |d|
    const size_t base = (((size_t)j * NB + nb) * KC + kc) * TC_TILE;
    for (int kb = t >> 7; kb < TC_KC / 8; kb += TC_THREADS / TC_N) {
        const int y0 = kc * (TC_KC / 2) + 4 * kb;
        uint32_t w0[4], w1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 p = make_float2(0.f, 0.f);
            if (col_ok) p = cmul(__ldg(Scol + (size_t)(y0 + i) * nx), __ldg(Ucol + (size_t)(y0 + i) * N));
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
        const size_t o = base + (tc_off(bn, 8 * kb) >> 1);
        *(uint4 *)(B0 + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        if (MODE == 1) *(uint4 *)(B1 + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    }
}

// ---------------------------------------------------------------- the GEMM

LRCCS_DEV void tc_bulk(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
LRCCS_DEV void tc_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// Stage layout: [A tiles: array a (0: hi / fp16, 1: lo), M tile m at
// (a MT + m)] then [B tiles: array a at a].  NA = 2 (BF16X3) or 1 (FP16S).
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_fwd_gemm(const uint16_t *__restrict__ A0,
                                                         const uint16_t *__restrict__ A1,
                                                         const uint16_t *__restrict__ B0,
                                                         const uint16_t *__restrict__ B1,
                                                         const int32_t *__restrict__ usedrows,
                                                         const float *__restrict__ tmax, float2 *__restrict__ T,
                                                         int ny, int nx, int r, int n_used, int mt, int tcols,
                                                         unsigned int *status) {
    constexpr int NA = MODE == 1 ? 2 : 1;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ __align__(8) uint64_t mbar[5];   // full[2], empty[2], done
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int t = threadIdx.x;
    const int nb = blockIdx.x, j = blockIdx.y, NB = gridDim.x;
    const int N = nx * r, K2 = 2 * ny, KC = K2 / TC_KC;
    const int mtiles_a = (2 * n_used + TC_M - 1) / TC_M;   // rows of A tiles (the A layout's bm stride)
    const uint32_t stage_bytes = (uint32_t)((NA * mt + NA) * TC_TILE_BYTES);
    uint32_t full[2], empty[2], done;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        full[i] = (uint32_t)__cvta_generic_to_shared(&mbar[i]);
        empty[i] = (uint32_t)__cvta_generic_to_shared(&mbar[2 + i]);
    }
    done = (uint32_t)__cvta_generic_to_shared(&mbar[4]);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tc_smem);
    if (t == 0) {
        for (int i = 0; i < 5; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(&mbar[i])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_fail = 0;
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_slot)),
                     "r"((uint32_t)tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    if (t == 0) {
        // producer: chunk kc into stage kc & 1, once the MMAs of chunk kc - 2 are done
        for (int kc = 0; kc < KC; ++kc) {
            const int st = kc & 1, use = kc >> 1;
            if (kc >= 2 && !tc_wait(empty[st], (uint32_t)((use - 1) & 1))) {
                atomicExch(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            tc_expect(full[st], stage_bytes);
            const uint32_t sst = sbase + st * stage_bytes;
            for (int a = 0; a < NA; ++a) {
                const uint16_t *Ag = a == 0 ? A0 : A1;
                for (int m = 0; m < mt; ++m)
                    tc_bulk(sst + (a * mt + m) * TC_TILE_BYTES, Ag + ((size_t)m * KC + kc) * TC_TILE, TC_TILE_BYTES,
                            full[st]);
                const uint16_t *Bg = a == 0 ? B0 : B1;
                tc_bulk(sst + (NA * mt + a) * TC_TILE_BYTES, Bg + (((size_t)j * NB + nb) * KC + kc) * TC_TILE,
                        TC_TILE_BYTES, full[st]);
            }
        }
    } else if (t == 32) {
        // MMA issuer
        const uint32_t idesc = tc_idesc(MODE == 1);
        int kc = 0;
        for (; kc < KC; ++kc) {
            const int st = kc & 1, use = kc >> 1;
            if (!tc_wait(full[st], (uint32_t)(use & 1))) {
                atomicExch(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sst = sbase + st * stage_bytes;
            const uint32_t b0 = sst + (NA * mt) * TC_TILE_BYTES, b1 = b0 + TC_TILE_BYTES;
            for (int m = 0; m < mt; ++m) {
                const uint32_t a0 = sst + m * TC_TILE_BYTES, a1 = sst + (mt + m) * TC_TILE_BYTES;
                const uint32_t acc_t = tmem + (uint32_t)(m * TC_N);
#pragma unroll
                for (int ks = 0; ks < TC_KC / 16; ++ks) {
                    const uint32_t ko = ks * 2 * 128;   // two K core matrices per MMA
                    tc_mma(acc_t, tc_desc(a0 + ko), tc_desc(b0 + ko), idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                    if (MODE == 1) {
                        tc_mma(acc_t, tc_desc(a0 + ko), tc_desc(b1 + ko), idesc, 1u);
                        tc_mma(acc_t, tc_desc(a1 + ko), tc_desc(b0 + ko), idesc, 1u);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                empty[st]));
        }
        // done: every MMA issued by this thread has completed (or nothing to wait for)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done));
    }
    // every thread: the accumulators are final
    bool ok = tc_wait(done, 0u);
    __syncthreads();
    // the producer's copies in flight (a failed run may leave some): wait
    // (bounded) for each stage's last arming before the block exits
    if (t == 0) {
        for (int kc = (KC >= 2 ? KC - 2 : 0); kc < KC; ++kc) tc_wait(full[kc & 1], (uint32_t)((kc >> 1) & 1));
    }
    ok = __syncthreads_and(ok && !s_fail);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const float binv = MODE == 2 ? 1.f / tile_scale(tmax[nb], tmax[-1]) : 1.f;
        // epilogue: warp w reads rows 32 (w % 4) .. + 31 (TMEM lanes), columns
        // 64 (w / 4) .. + 63 of each M tile's accumulator; the even lane of a
        // pair holds the real part of output row s, the odd lane its imaginary part
        const int w = t >> 5, lane = t & 31;
        const int row = 32 * (w & 3) + lane, cb = 64 * (w >> 2);
        const bool odd = lane & 1;
        const int n0 = nb * TC_N;
        for (int m = 0; m < mt; ++m) {
            const int s = (m * TC_M + row) >> 1;
            const int ky = s < n_used ? usedrows[s] : -1;
            float2 *Trow = T + ((size_t)j * ny + (ky < 0 ? 0 : ky)) * N;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(m * TC_N + cb + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
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
        }
    } else if (t == 0) {
        atomicOr(status, (unsigned)ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)tcols));
    (void)mtiles_a;
}

// ---------------------------------------------------------------- launchers

int tc_mtiles(int n_used) { return (2 * n_used + TC_M - 1) / TC_M; }
size_t tc_a_elems(int ny) { return (size_t)((2 * ny + TC_M - 1) / TC_M) * TC_M * 2 * ny; }   // per array, worst case
size_t tc_b_elems(int nc, int ny, int nx, int rmax) {   // per array
    return (size_t)nc * (((size_t)nx * rmax + TC_N - 1) / TC_N) * TC_N * 2 * ny;
}

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

static size_t gemm_smem(int mode, int mt, int tcols) {
    const int na = mode == 1 ? 2 : 1;
    size_t sm = (size_t)2 * (na * mt + na) * TC_TILE_BYTES;
    // keep the CTAs of one SM within its 512 tensor-memory columns
    const size_t floor_ = tcols >= 512 ? (size_t)120 * 1024 : tcols >= 256 ? (size_t)80 * 1024 : 0;
    return sm > floor_ ? sm : floor_;
}

cudaError_t launch_fwd_gemm(lrccs_ctx *c) {
    const int N = c->nx * c->r, NB = (N + TC_N - 1) / TC_N, KC = 2 * c->ny / TC_KC;
    const int mt = tc_mtiles(c->n_used);
    if (mt < 1 || mt > TC_MT_MAX) return cudaErrorInvalidValue;
    const int tcols = mt <= 1 ? 128 : (mt == 2 ? 256 : 512);
    cudaError_t e;
    if (c->dims.precision == LRCCS_PREC_FP16S_GEMM) {   // per-tile max |U| (d_tcscale[0] holds max |d|)
        prof_begin(c, KID_TC_SCALE);
        cudaMemsetAsync(c->d_tcscale + 1, 0, (size_t)NB * sizeof(float), c->stream);
        k_tile_max<<<dim3(NB, (c->ny + TS_ROWS - 1) / TS_ROWS), TC_N, 0, c->stream>>>(c->d_U, c->ny, N,
                                                                                    c->d_tcscale + 1);
        prof_end(c, KID_TC_SCALE);
    }
    const bool bf = c->dims.precision == LRCCS_PREC_BF16X3_GEMM;
    prof_begin(c, KID_TC_B);
    if (bf)
        k_b_operand<1><<<dim3(NB, KC, c->nc), TC_THREADS, 0, c->stream>>>(c->d_U, c->d_smaps, c->d_tcscale + 1,
                                                                          c->d_tcB0, c->d_tcB1, c->ny, c->nx, c->r);
    else
        k_b_operand<2><<<dim3(NB, KC, c->nc), TC_THREADS, 0, c->stream>>>(c->d_U, c->d_smaps, c->d_tcscale + 1,
                                                                          c->d_tcB0, c->d_tcB1, c->ny, c->nx, c->r);
    prof_end(c, KID_TC_B);
    prof_begin(c, KID_TC_GEMM);
    const size_t smem = gemm_smem(bf ? 1 : 2, mt, tcols);
    if (bf)
        k_fwd_gemm<1><<<dim3(NB, c->nc), TC_THREADS, smem, c->stream>>>(c->d_tcA0, c->d_tcA1, c->d_tcB0, c->d_tcB1,
                                                                        c->d_usedrows, c->d_tcscale + 1, c->d_T,
                                                                        c->ny, c->nx, c->r, c->n_used, mt, tcols,
                                                                        c->d_status);
    else
        k_fwd_gemm<2><<<dim3(NB, c->nc), TC_THREADS, smem, c->stream>>>(c->d_tcA0, c->d_tcA1, c->d_tcB0, c->d_tcB1,
                                                                        c->d_usedrows, c->d_tcscale + 1, c->d_T,
                                                                        c->ny, c->nx, c->r, c->n_used, mt, tcols,
                                                                        c->d_status);
    prof_end(c, KID_TC_GEMM);
    e = cudaGetLastError();
    return e;
}

cudaError_t configure_kernels_tc(int max_smem) {
    cudaError_t e = allow_smem(k_fwd_gemm<1>, max_smem);
    if (e == cudaSuccess) e = allow_smem(k_fwd_gemm<2>, max_smem);
    return e;
}
