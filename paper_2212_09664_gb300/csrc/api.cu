// api.cu -- the C ABI of liblrccs (declared in include/lrccs.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>

#include "internal.h"
#include "lrccs.h"

static std::string g_create_err;
static std::mutex g_err_mutex;   // the async worker and the caller's thread may both report errors

void set_err(lrccs_ctx *c, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    std::lock_guard<std::mutex> lock(g_err_mutex);
    if (c) c->err = buf;
    else g_create_err = buf;
}

cudaError_t configure_kernels_init(int max_smem);
cudaError_t configure_kernels_iter(int max_smem);
cudaError_t configure_kernels_gd(int max_smem);
cudaError_t configure_kernels_general(int max_smem);
cudaError_t configure_kernels_tc(int max_smem);
cudaError_t configure_kernels_zh(int max_smem);
cudaError_t configure_kernels_solve(int max_smem);

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_err(c, "%s failed: %s", #call, cudaGetErrorString(e_));                 \
            return LRCCS_E_CUDA;                                                        \
        }                                                                               \
    } while (0)

extern "C" void lrccs_default_params(lrccs_params *p) {
    if (!p) return;
    p->trunc_factor = 36.0;
    p->energy_pct = 85.0;
    p->eta_c = 0.14;
    p->eps_exit = 0.01;
    p->t_max = 70;
    p->exit_enabled = 0;
    p->admit_reserve_bytes = 268435456.0;
    p->exit_patience = 1;
    p->reserved = 0;
    p->eta_scale0 = 1.0;
    p->eta_decay = 1.0;
}

extern "C" const char *lrccs_status_string(lrccs_status s) {
    switch (s) {
        case LRCCS_OK: return "ok";
        case LRCCS_E_INVALID: return "invalid argument";
        case LRCCS_E_NOMEM: return "out of device memory";
        case LRCCS_E_CUDA: return "CUDA error";
        case LRCCS_E_RANK_DEFICIENT: return "rank deficient";
        case LRCCS_E_TIMEOUT: return "device wait timed out";
        case LRCCS_E_ADMISSION: return "admission refused";
        case LRCCS_E_STATE: return "call out of order";
        case LRCCS_E_UNSUPPORTED: return "unsupported input";
    }
    return "unknown status";
}

extern "C" const char *lrccs_last_error(const lrccs_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

static void free_all(lrccs_ctx *c) {
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    c->side = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    void *ptrs[] = {c->d_twy, c->d_twx, c->d_smaps, c->d_rowcnt, c->d_rowidx, c->d_framerows, c->d_lineptr,
                    c->d_rfptr, c->d_rflist, c->d_usedrows, c->d_rowused, c->d_idx, c->d_meta, c->d_status,
                    c->d_counters, c->d_scal, c->d_Z, c->d_X0, c->d_T, c->d_U, c->d_Uprev, c->d_Up, c->d_G,
                    c->d_B, c->d_P, c->d_gpart, c->d_sigma, c->d_gram, c->d_V, c->d_tot, c->d_framek,
                    c->d_mks, c->d_fpk, c->d_rowoff, c->d_ucnt, c->d_uloc, c->d_floc, c->d_urow, c->d_uptr,
                    c->d_ufrow, c->d_upos, c->d_uidx, c->d_ufptr, c->d_uflist, c->d_fu, c->d_FU, c->d_Pu,
                    c->d_maskc, c->d_mec, c->d_mscal, c->d_mout, c->d_twq, c->d_Q, c->d_gdts, c->d_fpart,
                    c->d_tflag, c->d_tcA0, c->d_tcA1, c->d_tcscale, c->d_ZB, c->d_hpart,
                    c->d_tcB0, c->d_tcB1};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <typename T>
static bool dalloc(lrccs_ctx *c, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "cudaMalloc(%zu bytes) failed: %s", count * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return false;
    }
    return true;
}

static bool pow_ok(int v) { return v >= 32 && v <= 256 && v % 32 == 0; }

static lrccs_status create_impl(const lrccs_dims *dims, const lrccs_params *params, void *cuda_stream,
                                lrccs_ctx **out, size_t *out_bytes_only) {
    if (!dims || (!out && !out_bytes_only)) {
        set_err(nullptr, "lrccs_create: dims and out must be non-null");
        return LRCCS_E_INVALID;
    }
    if (out) *out = nullptr;
    const lrccs_dims d = *dims;
    int rmax = d.rank_max > 0 ? d.rank_max : (d.rank > 0 ? d.rank : 16);
    if (!pow_ok(d.ny) || !pow_ok(d.nx) || d.q < 1 || d.q > 128 || d.ncoil < 1 || d.ncoil > 64 || d.rank < 0 ||
        d.rank > 16 || rmax < 1 || rmax > 16 || (d.rank > 0 && d.rank > rmax)) {
        set_err(nullptr,
                "lrccs_create: dims outside scope (ny, nx multiples of 32 in [32,256]; q in [1,128]; "
                "ncoil in [1,64]; 0 <= rank <= rank_max <= 16)");
        return LRCCS_E_INVALID;
    }
    if (d.precision != LRCCS_PREC_FP32_FFT && d.precision != LRCCS_PREC_BF16X3_GEMM &&
        d.precision != LRCCS_PREC_FP16S_GEMM) {
        set_err(nullptr, "lrccs_create: unknown precision %d", d.precision);
        return LRCCS_E_UNSUPPORTED;
    }
    lrccs_ctx *c = new (std::nothrow) lrccs_ctx();
    if (!c) return LRCCS_E_NOMEM;
    c->dims = d;
    if (params) c->prm = *params;
    else lrccs_default_params(&c->prm);
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->ny = d.ny;
    c->nx = d.nx;
    c->n = d.ny * d.nx;
    c->q = d.q;
    c->nc = d.ncoil;
    c->rmax = rmax;
    c->px = d.nx / 32;
    c->py = d.ny / 32;
    int nblk = (c->n + 127) / 128;
    if (nblk > 152) nblk = 152;
    c->nblk = nblk;
    const int n = c->n, q = c->q, nc = c->nc, ny = c->ny;
    const int npm = rmax * (rmax + 1) / 2;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int gd = (c->n + 31) / 32;
    if (gd > nsm) gd = nsm;
    if (gd < 1) gd = 1;
    c->gd_grid = gd;
    const size_t gd_len = std::max((size_t)2 * npm + rmax * rmax, (size_t)rmax * rmax + (size_t)q * rmax);
    size_t gcap = (size_t)gd * gd_len;
    if ((size_t)nblk * rmax * rmax > gcap) gcap = (size_t)nblk * rmax * rmax;
    if ((size_t)c->nx * npm > gcap) gcap = (size_t)c->nx * npm;
    if ((size_t)152 * q * (q + 1) / 2 > gcap) gcap = (size_t)152 * q * (q + 1) / 2;
    if (gcap < 1024) gcap = 1024;
    c->gpart_cap = gcap;
    c->T_cap = (size_t)nc * n * rmax;
    // every buffer of the context, as (pointer, bytes); the total is checked
    // against the free device memory before anything is allocated
    const size_t F2 = sizeof(float2), I4 = sizeof(int32_t), D8 = sizeof(double);
    const struct { void **p; size_t bytes; } plan[] = {
        {(void **)&c->d_twy, ny * F2}, {(void **)&c->d_twx, c->nx * F2}, {(void **)&c->d_smaps, (size_t)nc * n * F2},
        {(void **)&c->d_rowcnt, (size_t)q * ny * I4}, {(void **)&c->d_rowidx, (size_t)q * ny * I4},
        {(void **)&c->d_framerows, (size_t)q * ny * I4}, {(void **)&c->d_lineptr, ((size_t)q + 1) * I4},
        {(void **)&c->d_rfptr, ((size_t)ny + 1) * I4}, {(void **)&c->d_rflist, (size_t)q * ny * I4},
        {(void **)&c->d_usedrows, (size_t)ny * I4}, {(void **)&c->d_rowused, (size_t)ny},
        {(void **)&c->d_idx, (size_t)q * n * I4}, {(void **)&c->d_meta, ((size_t)MT_COUNT + q) * I4},
        {(void **)&c->d_status, sizeof(unsigned)}, {(void **)&c->d_counters, CNT_COUNT * sizeof(unsigned)},
        {(void **)&c->d_scal, SC_COUNT * D8}, {(void **)&c->d_Z, (size_t)n * q * F2},
        {(void **)&c->d_X0, (size_t)n * q * F2}, {(void **)&c->d_T, c->T_cap * F2},
        {(void **)&c->d_U, (size_t)n * rmax * F2}, {(void **)&c->d_Uprev, (size_t)n * rmax * F2},
        {(void **)&c->d_Up, (size_t)n * rmax * F2}, {(void **)&c->d_G, (size_t)n * rmax * F2},
        {(void **)&c->d_B, (size_t)q * rmax * F2}, {(void **)&c->d_P, (size_t)ny * npm * F2},
        {(void **)&c->d_gpart, gcap * F2}, {(void **)&c->d_tot, gd_len * sizeof(double2)},
        {(void **)&c->d_ZB, (size_t)n * rmax * F2}, {(void **)&c->d_hpart, (size_t)gd * q * rmax * F2},
        {(void **)&c->d_sigma, (size_t)q * D8}, {(void **)&c->d_gram, (size_t)6 * q * q * D8},
        {(void **)&c->d_V, (size_t)q * q * F2}, {(void **)&c->d_Q, (size_t)q * q * F2},
        {(void **)&c->d_framek, (size_t)q * ny * I4}, {(void **)&c->d_mks, (size_t)q * I4},
        {(void **)&c->d_fpk, ((size_t)q + 1) * I4}, {(void **)&c->d_rowoff, (size_t)q * ny * I4},
        {(void **)&c->d_maskc, (size_t)q * n}, {(void **)&c->d_twq, (size_t)q * F2},
        {(void **)&c->d_tcA0, d.precision != LRCCS_PREC_FP32_FFT ? tc_a_elems(ny) * 2 : 0},
        {(void **)&c->d_tcA1, d.precision == LRCCS_PREC_BF16X3_GEMM ? tc_a_elems(ny) * 2 : 0},
        {(void **)&c->d_tcB0, d.precision != LRCCS_PREC_FP32_FFT ? tc_b_elems(nc, ny, c->nx, rmax) * 2 : 0},
        {(void **)&c->d_tcB1, d.precision == LRCCS_PREC_BF16X3_GEMM ? tc_b_elems(nc, ny, c->nx, rmax) * 2 : 0},
        {(void **)&c->d_tcscale, (1 + ((size_t)c->nx * rmax + 127) / 128) * sizeof(float)},
    };
    size_t need = 0;
    for (const auto &it : plan) need += (it.bytes + 255) & ~(size_t)255;
    c->create_bytes = need;
    if (out_bytes_only) {
        *out_bytes_only = need;
        delete c;
        return LRCCS_OK;
    }
    // admission: the buffers must fit the free device memory with the reserve left over
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        set_err(nullptr, "lrccs_create: cudaMemGetInfo failed");
        delete c;
        return LRCCS_E_CUDA;
    }
    const double reserve = c->prm.admit_reserve_bytes > 0.0 ? c->prm.admit_reserve_bytes : 0.0;
    if ((double)need + reserve > (double)fr) {
        set_err(nullptr, "lrccs_create: admission refused: the context needs %zu bytes and %.0f must stay free, "
                         "but only %zu bytes of device memory are free", need, reserve, fr);
        delete c;
        return LRCCS_E_ADMISSION;
    }
    bool ok = true;
    for (const auto &it : plan) {
        *it.p = nullptr;
        if (ok) {
            cudaError_t e = cudaMalloc(it.p, it.bytes ? it.bytes : 1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_err(c, "cudaMalloc(%zu bytes) failed: %s", it.bytes, cudaGetErrorString(e));
                *it.p = nullptr;
                ok = false;
            }
        }
    }
    if (!ok) {
        g_create_err = c->err;
        free_all(c);
        delete c;
        return LRCCS_E_NOMEM;
    }
    int optin = 0, coop = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    c->dev_smem_optin = optin;
    cudaError_t e = configure_kernels_init(optin);
    if (e == cudaSuccess) e = configure_kernels_iter(optin);
    if (e == cudaSuccess) e = configure_kernels_gd(optin);
    if (e == cudaSuccess) e = configure_kernels_general(optin);
    if (e == cudaSuccess) e = configure_kernels_tc(optin);
    if (e == cudaSuccess) e = configure_kernels_zh(optin);
    if (e == cudaSuccess) e = configure_kernels_solve(optin);
    if (e == cudaSuccess) {
        c->nsm = nsm;
        for (int rr = 1; rr <= 16; ++rr) c->bs_cap[rr] = rr <= rmax ? bstep_capacity(nc, c->nx, q, rr, optin, nsm) : 0;
    }
    if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = launch_twiddles(c->d_twy, ny, c->stream);
    if (e == cudaSuccess) e = launch_twiddles(c->d_twx, c->nx, c->stream);
    if (e == cudaSuccess) e = launch_twiddles(c->d_twq, q, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, CNT_COUNT * sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_scal, 0, SC_COUNT * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_meta, 0, ((size_t)MT_COUNT + q) * sizeof(int32_t), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        set_err(nullptr, "lrccs_create: %s", cudaGetErrorString(e));
        free_all(c);
        delete c;
        return LRCCS_E_CUDA;
    }
    *out = c;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_create(const lrccs_dims *dims, const lrccs_params *params, void *cuda_stream,
                                     lrccs_ctx **out) {
    if (!out) {
        set_err(nullptr, "lrccs_create: dims and out must be non-null");
        return LRCCS_E_INVALID;
    }
    return create_impl(dims, params, cuda_stream, out, nullptr);
}

extern "C" lrccs_status lrccs_context_bytes(const lrccs_dims *dims, size_t *bytes) {
    if (!bytes) {
        set_err(nullptr, "lrccs_context_bytes: bytes must be non-null");
        return LRCCS_E_INVALID;
    }
    return create_impl(dims, nullptr, nullptr, nullptr, bytes);
}

static void drop_iter_graph(lrccs_ctx *c);

static void stop_worker(lrccs_ctx *c);

extern "C" void lrccs_destroy(lrccs_ctx *c) {
    if (!c) return;
    stop_worker(c);
    cudaStreamSynchronize(c->stream);
    for (const prof_rec &r : c->pending) {
        if (r.graph_owned) continue;   // owned by the graph, released below
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->pending.clear();
    drop_iter_graph(c);                // its events go back to the pool
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    c->event_pool.clear();
    free_all(c);
    delete c;
}

static lrccs_status status_to_code(lrccs_ctx *c, unsigned st) {
    if (st & ST_TIMEOUT) {   // first: a barrier that gave up explains any other flag
        set_err(c, "a bounded device wait timed out");
        return LRCCS_E_TIMEOUT;
    }
    if (st & ST_FRAMEPTR_MISMATCH) {
        set_err(c, "frame_ptr does not match the per-frame sample counts of the mask");
        return LRCCS_E_INVALID;
    }
    if (st & ST_ZERO_SIGMA) {
        set_err(c, "spectral initialisation: sigma_r(X0) = 0 or rank above rank_max");
        return LRCCS_E_RANK_DEFICIENT;
    }
    if (st & ST_NOT_SPD_LS) {
        set_err(c, "some frame's normal matrix (A_k U)^H (A_k U) is not positive definite");
        return LRCCS_E_RANK_DEFICIENT;
    }
    if (st & ST_NOT_SPD_QR) {
        set_err(c, "U + eta grad lost rank (CholeskyQR failed)");
        return LRCCS_E_RANK_DEFICIENT;
    }
    return LRCCS_OK;
}

static lrccs_status sync_status(lrccs_ctx *c) {
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return status_to_code(c, st);
}

// Buffers of the general-mask path (allocated the first time a context sees
// a mask with partly sampled rows).
static lrccs_status ensure_general_buffers(lrccs_ctx *c) {
    if (c->gen_cap_q) return LRCCS_OK;
    const size_t n = (size_t)c->n, q = (size_t)c->q, ny = (size_t)c->ny;
    const size_t npm = (size_t)c->rmax * (c->rmax + 1) / 2;
    const bool ok = dalloc(c, &c->d_ucnt, n) && dalloc(c, &c->d_uloc, n) && dalloc(c, &c->d_floc, n) &&
                    dalloc(c, &c->d_urow, 2 * ny) && dalloc(c, &c->d_uptr, ny + 1) &&
                    dalloc(c, &c->d_ufrow, ny + 1) && dalloc(c, &c->d_upos, n) && dalloc(c, &c->d_uidx, n) &&
                    dalloc(c, &c->d_ufptr, n + 1) && dalloc(c, &c->d_uflist, q * n) && dalloc(c, &c->d_fu, q * n) &&
                    dalloc(c, &c->d_FU, (size_t)c->nc * n * c->rmax) && dalloc(c, &c->d_Pu, n * npm) &&
                    dalloc(c, &c->d_fpart, frame_gram_part_count(c->q, c->rmax));
    if (!ok) return LRCCS_E_NOMEM;
    c->gen_cap_q = q;
    return LRCCS_OK;
}

// Mask compaction, the sampled-row structure and Z = [A_k^H y_k] for the data
// of one lrccs_init or tracking call; with_energy also forms gamma, which only
// the spectral initialisation's truncation uses.  Waits for the compaction's
// counts (twice for a general 2D mask: once for the row structure, once for
// the union of the frames' samples).
static lrccs_status load_data(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr, const uint8_t *d_mask,
                              const void *d_smaps, bool with_energy) {
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->d_counters, 0, CNT_COUNT * sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->d_meta, 0, MT_COUNT * sizeof(int32_t), c->stream));
    CK(cudaMemcpyAsync(c->d_smaps, d_smaps, (size_t)c->nc * c->n * sizeof(float2), cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_maskc, d_mask, (size_t)c->q * c->n, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_compact(c, d_mask, d_frame_ptr));
    lrccs_status s = sync_status(c);
    if (s != LRCCS_OK) return s;
    int32_t meta[MT_COUNT];
    CK(cudaMemcpy(meta, c->d_meta, sizeof(meta), cudaMemcpyDeviceToHost));
    c->n_used = meta[MT_NUSED];
    c->n_lines = meta[MT_NLINES];
    c->m_max = meta[MT_MMAX];
    c->total = meta[MT_TOTAL];
    c->general = meta[MT_GENERAL] ? 1 : 0;
    c->n_u = 0;
    if (c->total == 0 || c->n_used == 0) {
        set_err(c, "no sampled k-space");
        return LRCCS_E_INVALID;
    }
    if (c->general) {
        s = ensure_general_buffers(c);
        if (s != LRCCS_OK) return s;
        const size_t nflag = (size_t)c->nc * c->total;
        if (nflag > c->tflag_cap) {
            if (c->d_tflag) cudaFree(c->d_tflag);
            c->d_tflag = nullptr;
            c->tflag_cap = 0;
            if (!dalloc(c, &c->d_tflag, nflag)) return LRCCS_E_NOMEM;
            c->tflag_cap = nflag;
        }
        CK(launch_compact_general(c, d_mask));
        CK(cudaMemcpyAsync(meta, c->d_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->n_u = meta[MT_NU];
    } else {
        CK(launch_fill_lines(c));
    }
    if (c->dims.precision != LRCCS_PREC_FP32_FFT) CK(launch_dft_a(c));   // DFT rows of the sampled rows
    // line masks' init row pass: full rows (nx) for every (frame row, coil), plain
    // and truncated (the general masks' init needs no such buffer)
    const size_t need = c->general ? 0 : (size_t)2 * c->nc * c->n_lines * c->nx;
    if (need > c->T_cap) {
        cudaFree(c->d_T);
        c->d_T = nullptr;
        if (!dalloc(c, &c->d_T, need)) {
            c->T_cap = 0;
            return LRCCS_E_NOMEM;
        }
        c->T_cap = need;
    }
    if (with_energy) CK(launch_energy(c, (const float2 *)d_y));
    CK(launch_init_adjoint(c, (const float2 *)d_y));
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_init(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr, const uint8_t *d_mask,
                                   const void *d_smaps, int32_t *out_rank) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_y || !d_frame_ptr || !d_mask || !d_smaps) {
        set_err(c, "lrccs_init: null input pointer");
        return LRCCS_E_INVALID;
    }
    if (c->dims.rank > c->q) {   // U_0 = top-r left singular vectors of the n x q X0
        set_err(c, "lrccs_init: rank %d above q = %d (the spectral initialisation needs r <= q)", c->dims.rank, c->q);
        return LRCCS_E_INVALID;
    }
    c->initialized = 0;
    c->has_u = 0;
    c->need_h = 0;
    c->t = 0;
    CK(cudaMemsetAsync(c->d_scal, 0, SC_COUNT * sizeof(double), c->stream));
    lrccs_status s = load_data(c, d_y, d_frame_ptr, d_mask, d_smaps, true);
    if (s != LRCCS_OK) return s;
    CK(launch_gram_x0(c));
    if (c->dims.rank > 0 && c->dims.rank <= c->rmax) {
        // a fixed rank: the kernels after the eigensolver need no host decision,
        // so its status is read by the final synchronisation
        c->r = c->dims.rank;
    } else {
        s = sync_status(c);
        if (s != LRCCS_OK) return s;
        int32_t meta[MT_COUNT];
        CK(cudaMemcpy(meta, c->d_meta, sizeof(meta), cudaMemcpyDeviceToHost));
        c->r = meta[MT_RANK];
    }
    if (c->r < 1 || c->r > c->rmax) {
        set_err(c, "lrccs_init: rank %d outside [1, rank_max=%d]", c->r, c->rmax);
        return LRCCS_E_INVALID;
    }
    CK(launch_u0(c));
    CK(launch_gdqr(c, 0));
    CK(cudaMemcpyAsync(c->d_Uprev, c->d_U, (size_t)c->n * c->r * sizeof(float2), cudaMemcpyDeviceToDevice,
                       c->stream));
    s = sync_status(c);
    if (s != LRCCS_OK) return s;
    c->initialized = 1;
    c->has_u = 1;
    if (out_rank) *out_rank = c->r;
    return LRCCS_OK;
}

// U_0 <- the subspace in d_U (set from outside, or the previous mini-batch's
// final U): one Cholesky QR pass of it (the init mode of k_gdqr); the next
// B-step forms its right-hand sides U^H Z from the data now loaded.
static lrccs_status warm_start(lrccs_ctx *c) {
    const size_t ub = (size_t)c->n * c->r * sizeof(float2);
    CK(cudaMemcpyAsync(c->d_Up, c->d_U, ub, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_gdqr(c, 0));
    CK(cudaMemcpyAsync(c->d_Uprev, c->d_U, ub, cudaMemcpyDeviceToDevice, c->stream));
    c->need_h = 0;
    return LRCCS_OK;
}

// Capture n iterations (launch_iteration's kernels and, when kernels are being
// timed, their event records; nothing else) as one CUDA graph on the
// context's stream, cached per (n, timed kernels, rank, sampled rows, work
// buffer).  Returns false when the graph cannot be built here (the legacy
// default stream cannot be captured); the caller then launches directly.
static void drop_iter_graph(lrccs_ctx *c) {
    if (!c->iter_exec) return;
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->iter_exec);
    c->iter_exec = nullptr;
    if (c->iter_graph) cudaGraphDestroy(c->iter_graph);
    c->iter_graph = nullptr;
    for (const prof_rec &r : c->iter_prof) {
        c->event_pool.push_back(r.a);
        c->event_pool.push_back(r.b);
    }
    c->iter_prof.clear();
}

static bool graph_matches(const lrccs_ctx *c, int n_iter) {
    return c->iter_exec && c->iter_n == n_iter && c->iter_mask == c->prof_mask && c->iter_r == c->r &&
           c->iter_nused == c->n_used && c->iter_T == c->d_T && c->iter_general == c->general &&
           c->iter_nu == c->n_u;
}

static bool ensure_iter_graph(lrccs_ctx *c, int n_iter) {
    if (c->iter_graph_failed) return false;
    if (graph_matches(c, n_iter)) return true;
    if (c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread) {
        c->iter_graph_failed = true;
        return false;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;   // the caller is capturing this stream: launch into its capture
    }
    drop_iter_graph(c);
    if (c->prof_mask) {   // timing events are created now, not during the capture
        const size_t need = (size_t)2 * 8 * n_iter;
        while (c->event_pool.size() < need) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreate(&ev) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            c->event_pool.push_back(ev);
        }
    }
    long long before[KID_COUNT];
    memcpy(before, c->launches, sizeof(before));
    const size_t np0 = c->pending.size();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        c->capturing = true;
        cudaError_t el = cudaSuccess;
        for (int it = 0; it < n_iter && el == cudaSuccess; ++it) {
            c->capture_iter = it;   // timing events on captured iterations 8, 24, 40, ...
            el = launch_iteration(c);
        }
        c->capturing = false;
        e = cudaStreamEndCapture(c->stream, &g);
        if (el != cudaSuccess) e = el;
    }
    for (int k = 0; k < KID_COUNT; ++k) {
        c->iter_counts[k] = c->launches[k] - before[k];
        c->launches[k] = before[k];
    }
    for (size_t p = np0; p < c->pending.size(); ++p) {
        prof_rec r = c->pending[p];
        r.graph_owned = true;
        c->iter_prof.push_back(r);
    }
    c->pending.resize(np0);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->iter_exec, g, 0);
    if (e == cudaSuccess) {
        c->iter_graph = g;   // kept for batches (child graph nodes)
        ++c->iter_gen;
    } else if (g) {
        cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->iter_exec = nullptr;
        for (const prof_rec &r : c->iter_prof) {
            c->event_pool.push_back(r.a);
            c->event_pool.push_back(r.b);
        }
        c->iter_prof.clear();
        c->iter_graph_failed = true;
        return false;
    }
    c->iter_n = n_iter;
    c->iter_mask = c->prof_mask;
    c->iter_r = c->r;
    c->iter_nused = c->n_used;
    c->iter_T = c->d_T;
    c->iter_general = c->general;
    c->iter_nu = c->n_u;
    return true;
}

// n_iter iterations on the loaded data.  may_capture: build the iteration
// graph when none matches (lrccs_iterate); otherwise replay one only when it
// already matches (tracking calls, whose sampled rows change every call).
static lrccs_status run_iterations(lrccs_ctx *c, int n_iter, bool may_capture, lrccs_iter_info *info) {
    int exited = 0, passed = 0;
    const int patience = c->prm.exit_patience > 1 ? c->prm.exit_patience : 1;
    // without the per-iteration exit test, replay the captured n-iteration graph
    // (the same kernels, launched with fewer gaps); timing events, when
    // requested, are nodes of the graph and report its latest replay
    if (!c->prm.exit_enabled && n_iter > 1 &&
        (may_capture ? ensure_iter_graph(c, n_iter) : graph_matches(c, n_iter))) {
        CK(cudaGraphLaunch(c->iter_exec, c->stream));
        for (int k = 0; k < KID_COUNT; ++k) c->launches[k] += c->iter_counts[k];
        c->pending.insert(c->pending.end(), c->iter_prof.begin(), c->iter_prof.end());
        c->t += n_iter;
        n_iter = 0;
    }
    for (int it = 0; it < n_iter; ++it) {
        CK(launch_iteration(c));
        c->t += 1;
        if (c->prm.exit_enabled) {
            double sd = 0.0;
            CK(cudaMemcpyAsync(&sd, c->d_scal + SC_SD, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            passed = sd / sqrt((double)c->r) < c->prm.eps_exit ? passed + 1 : 0;
            if (passed >= patience) {
                exited = 1;
                break;
            }
        }
    }
    if (info || c->prm.exit_enabled) {
        lrccs_status s = sync_status(c);
        double sc[SC_COUNT];
        CK(cudaMemcpy(sc, c->d_scal, sizeof(sc), cudaMemcpyDeviceToHost));
        if (info) {
            info->t = c->t;
            info->exited = exited;
            info->eta = sc[SC_ETA];
            info->sd = sc[SC_SD];
            info->gnorm = sc[SC_GNORM];
        }
        return s;
    }
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_iterate(lrccs_ctx *c, int32_t n_iter, lrccs_iter_info *info) {
    if (!c) return LRCCS_E_INVALID;
    if (!c->initialized) {
        set_err(c, "lrccs_iterate: call lrccs_init first");
        return LRCCS_E_STATE;
    }
    if (n_iter < 0) {
        set_err(c, "lrccs_iterate: n_iter < 0");
        return LRCCS_E_INVALID;
    }
    if (c->need_h && n_iter > 0) {
        lrccs_status s = warm_start(c);
        if (s != LRCCS_OK) return s;
    }
    return run_iterations(c, n_iter, true, info);
}

// ---------------------------------------------------------------- subspace tracking (Alg. 4)

extern "C" lrccs_status lrccs_set_subspace(lrccs_ctx *c, const void *d_U, int32_t rank, double eta) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_U || rank < 1 || rank > c->rmax) {
        set_err(c, "lrccs_set_subspace: need d_U and 1 <= rank <= rank_max (%d)", c->rmax);
        return LRCCS_E_INVALID;
    }
    CK(cudaMemcpyAsync(c->d_U, d_U, (size_t)c->n * rank * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    const double eta_v = eta > 0.0 ? eta : 0.0, set_v = eta > 0.0 ? 1.0 : 0.0, zero = 0.0;
    CK(cudaMemcpyAsync(c->d_scal + SC_ETA, &eta_v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_ETASET, &set_v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_GNORM, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_TCNT, &zero, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->r = rank;
    c->t = 0;
    c->has_u = 1;
    c->need_h = 1;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_track_minibatch(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr,
                                              const uint8_t *d_mask, const void *d_smaps, int32_t t_max,
                                              int32_t reset_eta, void *d_X, lrccs_iter_info *info) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_y || !d_frame_ptr || !d_mask || !d_smaps || t_max < 1) {
        set_err(c, "lrccs_track_minibatch: null input pointer or t_max < 1");
        return LRCCS_E_INVALID;
    }
    if (!c->has_u) {
        set_err(c, "lrccs_track_minibatch: no subspace (lrccs_init, lrccs_set_subspace or lrccs_set_state first)");
        return LRCCS_E_STATE;
    }
    c->initialized = 0;
    // Alg. 4: the initialisation of Alg. 2 is replaced by U_0 <- U^(j-1)
    if (reset_eta) {
        CK(cudaMemsetAsync(c->d_scal + SC_ETASET, 0, sizeof(double), c->stream));
        CK(cudaMemsetAsync(c->d_scal + SC_TCNT, 0, sizeof(double), c->stream));
    }
    lrccs_status s = load_data(c, d_y, d_frame_ptr, d_mask, d_smaps, false);
    if (s != LRCCS_OK) return s;
    s = warm_start(c);
    if (s != LRCCS_OK) return s;
    c->t = 0;
    c->initialized = 1;
    s = run_iterations(c, t_max, false, info);
    if (s != LRCCS_OK) return s;
    if (d_X) CK(launch_images(c, (float2 *)d_X));
    return LRCCS_OK;
}

// ---------------------------------------------------------------- mean step (Alg. 1 steps 1 and 2a)

// CG on A^H A z = A^H y at rank 1 (the context's r is set to 1 by the caller).
static lrccs_status mean_cg(lrccs_ctx *c, const void *d_y, double tol, int max_iter, void *d_zbar, void *d_ytil,
                           int32_t *out_iters) {
    double *cg = (double *)c->d_tot;   // {gamma, alpha, stop}
    double h[3];
    CK(launch_cg_init(c, cg));
    CK(cudaMemcpyAsync(h, cg, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double norms0 = sqrt(h[0]);
    double gamma = h[0];
    int it = 0;
    while (it < max_iter && norms0 > 0.0 && sqrt(gamma) > tol * norms0) {
        CK(launch_normal_op(c));
        CK(launch_cg_step(c, cg));
        CK(cudaMemcpyAsync(h, cg, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (h[2] != 0.0) break;   // <p, A^H A p> <= 0: nothing left to reduce
        ++it;
        gamma = h[0];
    }
    const size_t zb = (size_t)c->n * sizeof(float2);
    CK(cudaMemcpyAsync(d_zbar, c->d_Uprev, zb, cudaMemcpyDeviceToDevice, c->stream));
    if (d_ytil) {
        CK(cudaMemcpyAsync(c->d_U, c->d_Uprev, zb, cudaMemcpyDeviceToDevice, c->stream));
        CK(launch_fwd_only(c));
        if (c->general) CK(launch_mean_resid_general(c, (const float2 *)d_y, (float2 *)d_ytil));
        else CK(launch_mean_resid(c, (const float2 *)d_y, (float2 *)d_ytil, c->m_max / c->nx));
    }
    lrccs_status s = sync_status(c);
    if (out_iters) *out_iters = it;
    return s;
}

extern "C" lrccs_status lrccs_mean_step(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr,
                                        const uint8_t *d_mask, const void *d_smaps, double tol, int32_t max_iter,
                                        void *d_zbar, void *d_ytil, int32_t *out_iters) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_y || !d_frame_ptr || !d_mask || !d_smaps || !d_zbar || !(tol >= 0.0) || max_iter < 0 ||
        max_iter > 10000) {
        set_err(c, "lrccs_mean_step: null pointer, tol < 0 or max_iter outside [0, 10000]");
        return LRCCS_E_INVALID;
    }
    if (d_ytil == d_y) {
        set_err(c, "lrccs_mean_step: d_ytil must not alias d_y");
        return LRCCS_E_INVALID;
    }
    // the CG vectors use the subspace buffers: the context holds no solve afterwards
    c->initialized = 0;
    c->has_u = 0;
    c->need_h = 0;
    c->t = 0;
    lrccs_status s = load_data(c, d_y, d_frame_ptr, d_mask, d_smaps, false);
    if (s != LRCCS_OK) return s;
    const int r_save = c->r;
    c->r = 1;
    s = mean_cg(c, d_y, tol, max_iter, d_zbar, d_ytil, out_iters);
    c->r = r_save;
    return s;
}

// ---------------------------------------------------------------- model-error correction (Alg. 3)

static lrccs_status mec_ensure(lrccs_ctx *c) {
    if (c->d_mec) return LRCCS_OK;
    const int w = c->rmax, nch = (c->q + w - 1) / w;
    if (!dalloc(c, &c->d_mec, (size_t)5 * nch * c->n * w) || !dalloc(c, &c->d_mscal, mec_scal_count(c->n, c->q, w)) ||
        !dalloc(c, &c->d_mout, 8)) {
        if (c->d_mec) cudaFree(c->d_mec);
        if (c->d_mscal) cudaFree(c->d_mscal);
        c->d_mec = nullptr;
        c->d_mscal = nullptr;
        return LRCCS_E_NOMEM;
    }
    c->mec_w = w;
    c->mec_nch = nch;
    return LRCCS_OK;
}

static float2 *mec_vec(lrccs_ctx *c, int which) {   // 0 E, 1 S, 2 P, 3 W, 4 M_prev
    return c->d_mec + (size_t)which * c->mec_nch * c->n * c->mec_w;
}

// dst = [N_k src_k]_k, chunk by chunk
static lrccs_status mec_normal(lrccs_ctx *c, const float2 *src, float2 *dst) {
    const size_t cs = (size_t)c->n * c->mec_w;
    for (int cc = 0; cc < c->mec_nch; ++cc)
        CK(launch_frame_normal_op(c, src + cc * cs, dst + cc * cs, c->mec_w, cc * c->mec_w));
    return LRCCS_OK;
}

// s_k = A_k^H ytt_k = Z[:, k] - N_k (U_{t-1} b_k) into S, P = S, E = 0, gamma_k = ||s_k||^2
static lrccs_status mec_start(lrccs_ctx *c) {
    float2 *P = mec_vec(c, 2), *W = mec_vec(c, 3);
    CK(launch_mec_x(c, c->d_Uprev, nullptr, P));
    lrccs_status s = mec_normal(c, P, W);
    if (s != LRCCS_OK) return s;
    CK(launch_mec_cg(c, 0, W));
    return LRCCS_OK;
}

// `iters` CGLS iterations per frame (normal-equation form) from e = 0
static lrccs_status mec1_run(lrccs_ctx *c, int iters) {
    lrccs_status s = mec_start(c);
    if (s != LRCCS_OK) return s;
    for (int it = 0; it < iters; ++it) {
        s = mec_normal(c, mec_vec(c, 2), mec_vec(c, 3));   // W = N P
        if (s != LRCCS_OK) return s;
        CK(launch_mec_cg(c, 1, nullptr));   // alpha
        CK(launch_mec_cg(c, 2, nullptr));   // E, S, beta
        CK(launch_mec_cg(c, 3, nullptr));   // P
    }
    return LRCCS_OK;
}

static lrccs_status mec_check(lrccs_ctx *c, const char *who) {
    if (!c->initialized || c->t < 1 || c->need_h) {
        set_err(c, "%s: run at least one iteration (or an online call) first", who);
        return LRCCS_E_STATE;
    }
    return mec_ensure(c);
}

extern "C" lrccs_status lrccs_mec1(lrccs_ctx *c, int32_t iters, const void *d_zbar, void *d_E, void *d_X) {
    if (!c) return LRCCS_E_INVALID;
    if (iters < 0 || iters > 1000) {
        set_err(c, "lrccs_mec1: iters outside [0, 1000]");
        return LRCCS_E_INVALID;
    }
    lrccs_status s = mec_check(c, "lrccs_mec1");
    if (s != LRCCS_OK) return s;
    s = mec1_run(c, iters);
    if (s != LRCCS_OK) return s;
    CK(launch_mec_out(c, mec_vec(c, 0), (const float2 *)d_zbar, (float2 *)d_E, (float2 *)d_X));
    return sync_status(c);
}

extern "C" lrccs_status lrccs_mec2(lrccs_ctx *c, int32_t max_iter, double rel_change, double omega_frac,
                                   const void *d_zbar, void *d_E, void *d_X, int32_t *out_iters) {
    if (!c) return LRCCS_E_INVALID;
    if (max_iter < 0 || max_iter > 1000 || !(rel_change >= 0.0) || !(omega_frac >= 0.0)) {
        set_err(c, "lrccs_mec2: max_iter outside [0, 1000], or a negative rel_change / omega_frac");
        return LRCCS_E_INVALID;
    }
    lrccs_status s = mec_check(c, "lrccs_mec2");
    if (s != LRCCS_OK) return s;
    s = mec_start(c);   // S = s_0 = A^H ytt, E = 0
    if (s != LRCCS_OK) return s;
    float2 *E = mec_vec(c, 0), *S0 = mec_vec(c, 1), *V = mec_vec(c, 3);
    float2 *M = mec_vec(c, 2), *Mprev = mec_vec(c, 4);
    double omega = 0.0, h[3];
    int tau = 0;
    while (tau < max_iter) {
        if (tau > 0) {   // V = N E (E = 0 at tau = 0)
            s = mec_normal(c, E, V);
            if (s != LRCCS_OK) return s;
        }
        CK(launch_tdft_fwd(c, E, S0, tau > 0 ? V : nullptr, tau > 0 ? Mprev : nullptr, M, c->d_mout));
        CK(cudaMemcpyAsync(h, c->d_mout, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (tau == 0) omega = omega_frac * h[0];
        else if (sqrt(h[1]) < rel_change * sqrt(h[2])) break;
        CK(launch_tdft_inv(c, M, (float)omega, E));
        float2 *t = M;
        M = Mprev;
        Mprev = t;
        ++tau;
    }
    if (out_iters) *out_iters = tau;
    CK(launch_mec_out(c, E, (const float2 *)d_zbar, (float2 *)d_E, (float2 *)d_X));
    return sync_status(c);
}

// ---------------------------------------------------------------- online subspace tracking (Alg. 5)

extern "C" lrccs_status lrccs_online_frames(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr,
                                            const uint8_t *d_mask, const void *d_smaps, const void *d_zbar,
                                            int32_t mec_iters, void *d_X, void *d_B) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_y || !d_frame_ptr || !d_mask || !d_smaps || !d_zbar || mec_iters < 0 || mec_iters > 1000) {
        set_err(c, "lrccs_online_frames: null input pointer or mec_iters outside [0, 1000]");
        return LRCCS_E_INVALID;
    }
    if (!c->has_u) {
        set_err(c, "lrccs_online_frames: no subspace (lrccs_set_subspace or lrccs_set_state first)");
        return LRCCS_E_STATE;
    }
    c->initialized = 0;
    lrccs_status s = load_data(c, d_y, d_frame_ptr, d_mask, d_smaps, false);
    if (s != LRCCS_OK) return s;
    s = mec_ensure(c);
    if (s != LRCCS_OK) return s;
    // A_k^H y~_k = Z[:, k] - N_k zbar  (y~_k = y_k - A_k zbar)
    float2 *P = mec_vec(c, 2), *W = mec_vec(c, 3);
    CK(launch_mec_x(c, nullptr, (const float2 *)d_zbar, P));
    s = mec_normal(c, P, W);
    if (s != LRCCS_OK) return s;
    CK(launch_mec_subz(c, W));
    // U fixed: re-orthonormalise it (rounding only), h_k = U^H A_k^H y~_k, and the B-step
    s = warm_start(c);
    if (s != LRCCS_OK) return s;
    CK(launch_bstep(c));
    c->t = 1;
    c->initialized = 1;
    // MEC-1 on ytt_k = y~_k - A_k U b_k, then x_k = zbar + U b_k + e_k
    s = mec1_run(c, mec_iters);
    if (s != LRCCS_OK) return s;
    CK(launch_mec_out(c, mec_vec(c, 0), (const float2 *)d_zbar, nullptr, (float2 *)d_X));
    if (d_B) CK(cudaMemcpyAsync(d_B, c->d_B, (size_t)c->q * c->r * sizeof(float2), cudaMemcpyDeviceToDevice,
                                c->stream));
    return sync_status(c);
}

// ---------------------------------------------------------------- asynchronous tracking requests

#define ASYNC_SLOTS 256   // results (status, event, device status word) of the last 256 requests

struct track_req {
    uint64_t id;
    const void *y;
    const int64_t *fp;
    const uint8_t *mask;
    const void *smaps;
    int t_max, reset_eta;
    void *X;
};

struct async_worker {
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_req, cv_done;
    std::deque<track_req> queue;
    bool stop = false;
    uint64_t next_id = 1, done_id = 0;    // requests run in id order
    uint64_t slot_id[ASYNC_SLOTS] = {};
    lrccs_status slot_st[ASYNC_SLOTS] = {};
    cudaEvent_t slot_ev[ASYNC_SLOTS] = {};
    unsigned *slot_dev_status = nullptr;  // pinned host words, one per slot
};

static void worker_main(lrccs_ctx *c) {
    async_worker *w = c->worker;
    cudaSetDevice(c->device);
    for (;;) {
        track_req r;
        {
            std::unique_lock<std::mutex> lock(w->mu);
            w->cv_req.wait(lock, [&] { return w->stop || !w->queue.empty(); });
            if (w->queue.empty()) return;   // stop requested and nothing left
            r = w->queue.front();
            w->queue.pop_front();
        }
        const int sl = (int)(r.id % ASYNC_SLOTS);
        lrccs_status st =
            lrccs_track_minibatch(c, r.y, r.fp, r.mask, r.smaps, r.t_max, r.reset_eta, r.X, nullptr);
        if (st == LRCCS_OK) {
            // the request's device status word, read back behind its kernels
            if (cudaMemcpyAsync(w->slot_dev_status + sl, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaEventRecord(w->slot_ev[sl], c->stream) != cudaSuccess) {
                cudaGetLastError();
                st = LRCCS_E_CUDA;
            }
        }
        {
            std::lock_guard<std::mutex> lock(w->mu);
            w->slot_id[sl] = r.id;
            w->slot_st[sl] = st;
            w->done_id = r.id;
        }
        w->cv_done.notify_all();
    }
}

static lrccs_status start_worker(lrccs_ctx *c) {
    if (c->worker) return LRCCS_OK;
    async_worker *w = new (std::nothrow) async_worker();
    if (!w) return LRCCS_E_NOMEM;
    if (cudaHostAlloc((void **)&w->slot_dev_status, ASYNC_SLOTS * sizeof(unsigned), cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        delete w;
        set_err(c, "lrccs_track_minibatch_async: cudaHostAlloc failed");
        return LRCCS_E_CUDA;
    }
    for (int i = 0; i < ASYNC_SLOTS; ++i) {
        if (cudaEventCreateWithFlags(&w->slot_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) cudaEventDestroy(w->slot_ev[j]);
            cudaFreeHost(w->slot_dev_status);
            delete w;
            set_err(c, "lrccs_track_minibatch_async: cudaEventCreate failed");
            return LRCCS_E_CUDA;
        }
    }
    c->worker = w;
    w->th = std::thread(worker_main, c);
    return LRCCS_OK;
}

static void stop_worker(lrccs_ctx *c) {
    async_worker *w = c->worker;
    if (!w) return;
    {
        std::lock_guard<std::mutex> lock(w->mu);
        w->stop = true;
    }
    w->cv_req.notify_all();
    if (w->th.joinable()) w->th.join();
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < ASYNC_SLOTS; ++i) cudaEventDestroy(w->slot_ev[i]);
    cudaFreeHost(w->slot_dev_status);
    delete w;
    c->worker = nullptr;
}

extern "C" lrccs_status lrccs_track_minibatch_async(lrccs_ctx *c, const void *d_y, const int64_t *d_frame_ptr,
                                                    const uint8_t *d_mask, const void *d_smaps, int32_t t_max,
                                                    int32_t reset_eta, void *d_X, lrccs_ticket *ticket) {
    if (!c) return LRCCS_E_INVALID;
    if (!d_y || !d_frame_ptr || !d_mask || !d_smaps || !ticket || t_max < 1) {
        set_err(c, "lrccs_track_minibatch_async: null pointer or t_max < 1");
        return LRCCS_E_INVALID;
    }
    lrccs_status s = start_worker(c);
    if (s != LRCCS_OK) return s;
    async_worker *w = c->worker;
    {
        std::lock_guard<std::mutex> lock(w->mu);
        track_req r;
        r.id = w->next_id++;
        r.y = d_y;
        r.fp = d_frame_ptr;
        r.mask = d_mask;
        r.smaps = d_smaps;
        r.t_max = t_max;
        r.reset_eta = reset_eta;
        r.X = d_X;
        w->queue.push_back(r);
        ticket->id = r.id;
    }
    w->cv_req.notify_one();
    return LRCCS_OK;
}

// The slot of a ticket that has run, or -1 (expired / unknown); w->mu held.
static int ticket_slot(async_worker *w, uint64_t id) {
    const int sl = (int)(id % ASYNC_SLOTS);
    return (id >= 1 && w->slot_id[sl] == id) ? sl : -1;
}

extern "C" lrccs_status lrccs_ticket_query(lrccs_ctx *c, const lrccs_ticket *t, int32_t *done) {
    if (!c || !t || !done) return LRCCS_E_INVALID;
    async_worker *w = c->worker;
    if (!w || t->id < 1) {
        set_err(c, "lrccs_ticket_query: unknown ticket");
        return LRCCS_E_STATE;
    }
    std::unique_lock<std::mutex> lock(w->mu);
    if (t->id >= w->next_id) {
        set_err(c, "lrccs_ticket_query: unknown ticket");
        return LRCCS_E_STATE;
    }
    if (t->id > w->done_id) {
        *done = 0;
        return LRCCS_OK;
    }
    const int sl = ticket_slot(w, t->id);
    if (sl < 0) {
        set_err(c, "lrccs_ticket_query: expired ticket (results of the last %d requests are kept)", ASYNC_SLOTS);
        return LRCCS_E_STATE;
    }
    const lrccs_status st = w->slot_st[sl];
    cudaEvent_t ev = w->slot_ev[sl];
    lock.unlock();
    if (st != LRCCS_OK) {
        *done = 1;
        return st;
    }
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        *done = 0;
        return LRCCS_OK;
    }
    *done = 1;
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "lrccs_ticket_query: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    return status_to_code(c, w->slot_dev_status[sl]);
}

extern "C" lrccs_status lrccs_ticket_wait(lrccs_ctx *c, const lrccs_ticket *t) {
    if (!c || !t) return LRCCS_E_INVALID;
    async_worker *w = c->worker;
    if (!w || t->id < 1) {
        set_err(c, "lrccs_ticket_wait: unknown ticket");
        return LRCCS_E_STATE;
    }
    std::unique_lock<std::mutex> lock(w->mu);
    if (t->id >= w->next_id) {
        set_err(c, "lrccs_ticket_wait: unknown ticket");
        return LRCCS_E_STATE;
    }
    w->cv_done.wait(lock, [&] { return w->done_id >= t->id; });
    const int sl = ticket_slot(w, t->id);
    if (sl < 0) {
        set_err(c, "lrccs_ticket_wait: expired ticket (results of the last %d requests are kept)", ASYNC_SLOTS);
        return LRCCS_E_STATE;
    }
    const lrccs_status st = w->slot_st[sl];
    cudaEvent_t ev = w->slot_ev[sl];
    lock.unlock();
    if (st != LRCCS_OK) return st;
    const cudaError_t e = cudaEventSynchronize(ev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "lrccs_ticket_wait: %s", cudaGetErrorString(e));
        return LRCCS_E_CUDA;
    }
    return status_to_code(c, w->slot_dev_status[sl]);
}

// State buffer: this header, then U (n x r complex64).
struct state_header {
    uint32_t magic, version;
    int32_t ny, nx, r, t, eta_set, tcnt;   // tcnt: iterations since eta was set (step-size schedule)
    double eta, gnorm;
    uint8_t pad[16];
};
static_assert(sizeof(state_header) == 64, "state header is 64 bytes");
static const uint32_t kStateMagic = 0x5343524Cu;   // "LRCS"

extern "C" lrccs_status lrccs_get_state(lrccs_ctx *c, void *host_buf, size_t *bytes) {
    if (!c) return LRCCS_E_INVALID;
    if (!bytes) {
        set_err(c, "lrccs_get_state: bytes must be non-null");
        return LRCCS_E_INVALID;
    }
    if (!c->has_u) {
        set_err(c, "lrccs_get_state: no subspace yet");
        return LRCCS_E_STATE;
    }
    const size_t ub = (size_t)c->n * c->r * sizeof(float2);
    const size_t need = sizeof(state_header) + ub;
    if (!host_buf) {
        *bytes = need;
        return LRCCS_OK;
    }
    if (*bytes < need) {
        set_err(c, "lrccs_get_state: buffer holds %zu bytes, %zu needed", *bytes, need);
        return LRCCS_E_INVALID;
    }
    double sc[SC_COUNT];
    CK(cudaMemcpyAsync(sc, c->d_scal, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync((char *)host_buf + sizeof(state_header), c->d_U, ub, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    state_header h;
    memset(&h, 0, sizeof(h));
    h.magic = kStateMagic;
    h.version = 1;
    h.ny = c->ny;
    h.nx = c->nx;
    h.r = c->r;
    h.t = c->t;
    h.eta_set = sc[SC_ETASET] != 0.0 ? 1 : 0;
    h.tcnt = (int32_t)sc[SC_TCNT];
    h.eta = sc[SC_ETA];
    h.gnorm = sc[SC_GNORM];
    memcpy(host_buf, &h, sizeof(h));
    *bytes = need;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_set_state(lrccs_ctx *c, const void *host_buf, size_t bytes) {
    if (!c) return LRCCS_E_INVALID;
    if (!host_buf || bytes < sizeof(state_header)) {
        set_err(c, "lrccs_set_state: null or short buffer");
        return LRCCS_E_INVALID;
    }
    state_header h;
    memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1) {
        set_err(c, "lrccs_set_state: not a state buffer of this library");
        return LRCCS_E_INVALID;
    }
    if (h.ny != c->ny || h.nx != c->nx || h.r < 1 || h.r > c->rmax || h.t < 0) {
        set_err(c, "lrccs_set_state: state of a %dx%d rank-%d solve does not fit this context (%dx%d, rank_max %d)",
                h.ny, h.nx, h.r, c->ny, c->nx, c->rmax);
        return LRCCS_E_INVALID;
    }
    const size_t ub = (size_t)c->n * h.r * sizeof(float2);
    if (bytes < sizeof(state_header) + ub) {
        set_err(c, "lrccs_set_state: buffer holds %zu bytes, %zu needed", bytes, sizeof(state_header) + ub);
        return LRCCS_E_INVALID;
    }
    const double set_v = h.eta_set ? 1.0 : 0.0, tcnt_v = h.tcnt > 0 ? (double)h.tcnt : 0.0;
    CK(cudaMemcpyAsync(c->d_U, (const char *)host_buf + sizeof(state_header), ub, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_ETA, &h.eta, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_GNORM, &h.gnorm, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_ETASET, &set_v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_scal + SC_TCNT, &tcnt_v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->r = h.r;
    c->t = h.t;
    c->has_u = 1;
    c->need_h = 1;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_get_factors(lrccs_ctx *c, void *d_U, void *d_B) {
    if (!c) return LRCCS_E_INVALID;
    if (!c->initialized || c->need_h) {
        set_err(c, "lrccs_get_factors: no factors (call lrccs_init, or iterate after setting the subspace)");
        return LRCCS_E_STATE;
    }
    if (d_U)
        CK(cudaMemcpyAsync(d_U, c->d_Uprev, (size_t)c->n * c->r * sizeof(float2), cudaMemcpyDeviceToDevice,
                           c->stream));
    if (d_B && c->t > 0)
        CK(cudaMemcpyAsync(d_B, c->d_B, (size_t)c->q * c->r * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_get_subspace(lrccs_ctx *c, void *d_U) {
    if (!c || !d_U) return LRCCS_E_INVALID;
    if (!c->has_u) {
        set_err(c, "lrccs_get_subspace: no subspace yet");
        return LRCCS_E_STATE;
    }
    CK(cudaMemcpyAsync(d_U, c->d_U, (size_t)c->n * c->r * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_get_images(lrccs_ctx *c, void *d_X) {
    if (!c || !d_X) return LRCCS_E_INVALID;
    if (!c->initialized || c->t == 0 || c->need_h) {
        set_err(c, "lrccs_get_images: run at least one iteration first");
        return LRCCS_E_STATE;
    }
    CK(launch_images(c, (float2 *)d_X));
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_get_buffer(lrccs_ctx *c, lrccs_buffer which, void *d_dst, size_t bytes) {
    if (!c || !d_dst) return LRCCS_E_INVALID;
    const void *src = nullptr;
    size_t sz = 0;
    switch (which) {
        case LRCCS_BUF_Z: src = c->d_Z; sz = (size_t)c->n * c->q * sizeof(float2); break;
        case LRCCS_BUF_X0: src = c->d_X0; sz = (size_t)c->n * c->q * sizeof(float2); break;
        case LRCCS_BUF_GRAD: src = c->d_G; sz = (size_t)c->n * (c->r ? c->r : c->rmax) * sizeof(float2); break;
        case LRCCS_BUF_SIGMA: src = c->d_sigma; sz = (size_t)c->q * sizeof(double); break;
        case LRCCS_BUF_IDX: src = c->d_idx; sz = (size_t)c->total * sizeof(int32_t); break;
        case LRCCS_BUF_SCAL: src = c->d_scal; sz = SC_COUNT * sizeof(double); break;
        default: set_err(c, "lrccs_get_buffer: unknown buffer"); return LRCCS_E_INVALID;
    }
    if (bytes < sz) {
        set_err(c, "lrccs_get_buffer: destination holds %zu bytes, %zu needed", bytes, sz);
        return LRCCS_E_INVALID;
    }
    if (sz) CK(cudaMemcpyAsync(d_dst, src, sz, cudaMemcpyDeviceToDevice, c->stream));
    return LRCCS_OK;
}

// ---------------------------------------------------------------- profiling

const char *const kKernelNames[KID_COUNT] = {
    "k_rowcount", "k_structure", "k_fill_idx", "k_energy", "k_init_rows", "k_init_cols", "k_gram_x0",
    "k_eig", "k_u0", "k_gdqr", "k_fwd_cols", "k_row_gram", "k_solve", "k_row_w", "k_adj_cols",
    "k_images", "k_cg_init", "k_cg_step", "k_mean_resid", "k_union", "k_fill_general", "k_init_gen",
    "k_fwd_rows", "k_sample_gram", "k_solve_gen", "k_sample_w", "k_adj_rows", "k_mean_resid_gen", "k_mec_mask",
    "k_mec_elem", "k_mec_tdft", "k_dft_a", "k_fwd_gemm", "k_tile_max", "k_b_operand", "k_zb", "k_bstep"};

static cudaEvent_t get_event(lrccs_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(lrccs_ctx *c, int kid) {
    c->launches[kid] += 1;
    c->prof_this = (c->prof_mask & (1ull << kid)) && !(c->capturing && (c->capture_iter & 15) != 8);
    if (c->prof_this) {
        prof_rec r;
        r.kid = kid;
        r.graph_owned = false;
        r.a = get_event(c);
        r.b = get_event(c);
        // while the library captures its iteration graph the record must be
        // External to become an event-record node (a plain record there only
        // orders the capture); outside a capture it is a plain record
        if (c->capturing) cudaEventRecordWithFlags(r.a, c->stream, cudaEventRecordExternal);
        else cudaEventRecord(r.a, c->stream);
        c->pending.push_back(r);
    }
}

void prof_end(lrccs_ctx *c, int kid) {
    if (c->prof_this && !c->pending.empty()) {
        if (c->capturing) cudaEventRecordWithFlags(c->pending.back().b, c->stream, cudaEventRecordExternal);
        else cudaEventRecord(c->pending.back().b, c->stream);
    }
}

static lrccs_status prof_fold(lrccs_ctx *c) {
    CK(cudaStreamSynchronize(c->stream));
    for (const prof_rec &r : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.kid] += ms;
            c->timed[r.kid] += 1;
        } else {
            cudaGetLastError();   // an unreadable pair is skipped, not reported later
        }
        if (!r.graph_owned) {
            c->event_pool.push_back(r.a);
            c->event_pool.push_back(r.b);
        }
    }
    c->pending.clear();
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_profile(lrccs_ctx *c, const char *pattern) {
    if (!c) return LRCCS_E_INVALID;
    unsigned long long m = 0;
    if (pattern && *pattern) {
        for (int k = 0; k < KID_COUNT; ++k)
            if (!strcmp(pattern, "*") || strstr(kKernelNames[k], pattern)) m |= 1ull << k;
    }
    c->prof_mask = m;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_profile_read(lrccs_ctx *c, lrccs_kernel_stat *out, int32_t max, int32_t *count) {
    if (!c) return LRCCS_E_INVALID;
    lrccs_status s = prof_fold(c);
    if (s != LRCCS_OK) return s;
    for (int k = 0; k < KID_COUNT && k < max && out; ++k) {
        out[k].name = kKernelNames[k];
        out[k].launches = c->launches[k];
        out[k].timed = c->timed[k];
        out[k].ms = c->prof_ms[k];
    }
    if (count) *count = KID_COUNT;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_profile_reset(lrccs_ctx *c) {
    if (!c) return LRCCS_E_INVALID;
    lrccs_status s = prof_fold(c);
    for (int k = 0; k < KID_COUNT; ++k) {
        c->launches[k] = 0;
        c->timed[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    return s;
}

// ---------------------------------------------------------------- launch plan and autotuner

extern "C" lrccs_status lrccs_set_plan(lrccs_ctx *c, const lrccs_plan *plan) {
    if (!c || !plan) return LRCCS_E_INVALID;
    c->plan = *plan;
    drop_iter_graph(c);
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_get_plan(lrccs_ctx *c, lrccs_plan *plan) {
    if (!c || !plan) return LRCCS_E_INVALID;
    *plan = c->plan;
    return LRCCS_OK;
}

// The solver state one iteration reads and writes: U_t, U_{t-1}, B, the
// scalars (step size, its schedule counter, SD), the k_gdqr totals and its
// partial sums of the next right-hand sides U^H Z.
struct solver_state {
    std::vector<float2> U, Up, B, hpart;
    std::vector<double> scal;
    std::vector<double2> tot;
    int t;
};
static lrccs_status save_state(lrccs_ctx *c, solver_state &s, size_t tot_len) {
    const size_t nu = (size_t)c->n * c->r;
    s.U.resize(nu);
    s.Up.resize(nu);
    s.B.resize((size_t)c->q * c->r);
    s.scal.resize(SC_COUNT);
    s.tot.resize(tot_len);
    s.hpart.resize((size_t)c->gd_grid * c->q * c->r);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(s.hpart.data(), c->d_hpart, s.hpart.size() * sizeof(float2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.U.data(), c->d_U, nu * sizeof(float2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.Up.data(), c->d_Uprev, nu * sizeof(float2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.B.data(), c->d_B, s.B.size() * sizeof(float2), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.scal.data(), c->d_scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.tot.data(), c->d_tot, tot_len * sizeof(double2), cudaMemcpyDeviceToHost));
    s.t = c->t;
    return LRCCS_OK;
}
static lrccs_status restore_state(lrccs_ctx *c, const solver_state &s) {
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(c->d_U, s.U.data(), s.U.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_Uprev, s.Up.data(), s.Up.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_B, s.B.data(), s.B.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_scal, s.scal.data(), SC_COUNT * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_tot, s.tot.data(), s.tot.size() * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_hpart, s.hpart.data(), s.hpart.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemset(c->d_status, 0, sizeof(unsigned)));
    c->t = s.t;
    return LRCCS_OK;
}

// Best of two timed runs of n_iter directly launched iterations under `plan`
// (ms), from the saved state; < 0 if a launch of the plan failed.
static double time_plan(lrccs_ctx *c, const lrccs_plan &plan, int n_iter, const solver_state &st) {
    c->plan = plan;
    double best = -1.0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    for (int rep = 0; rep < 2; ++rep) {
        if (restore_state(c, st) != LRCCS_OK) break;
        cudaEventRecord(a, c->stream);
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < n_iter && e == cudaSuccess; ++i) e = launch_iteration(c);
        cudaEventRecord(b, c->stream);
        if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
            cudaGetLastError();
            best = -1.0;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best < 0.0 || ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

extern "C" lrccs_status lrccs_autotune(lrccs_ctx *c, int32_t n_iter, const char *cache_path, lrccs_plan *out) {
    if (!c) return LRCCS_E_INVALID;
    if (!c->initialized || c->need_h) {
        set_err(c, "lrccs_autotune: load data first (lrccs_init)");
        return LRCCS_E_STATE;
    }
    if (n_iter < 1) n_iter = 1;
    if (n_iter > 100) n_iter = 100;
    char key[160];
    snprintf(key, sizeof(key), "%d %d %d %d %d %d %d", c->ny, c->nx, c->q, c->nc, c->r, c->general,
             c->dims.precision);
    if (cache_path) {   // a tuned plan of this shape: apply it
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[256];
            bool found = false;
            while (fgets(line, sizeof(line), f)) {
                lrccs_plan pl = {};
                int v[7];
                if (sscanf(line, "%d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                           &pl.fwd_tx, &pl.coil_groups, &pl.row_groups) == 10) {
                    char k2[160];
                    snprintf(k2, sizeof(k2), "%d %d %d %d %d %d %d", v[0], v[1], v[2], v[3], v[4], v[5], v[6]);
                    if (!strcmp(k2, key)) {
                        c->plan = pl;
                        found = true;
                    }
                }
            }
            fclose(f);
            if (found) {
                drop_iter_graph(c);
                if (out) *out = c->plan;
                return LRCCS_OK;
            }
        }
    }
    const int npm = c->rmax * (c->rmax + 1) / 2;
    const size_t tot_len = std::max((size_t)2 * npm + (size_t)c->rmax * c->rmax,
                                    (size_t)c->rmax * c->rmax + (size_t)c->q * c->rmax);
    solver_state st;
    lrccs_status s = save_state(c, st, tot_len);
    if (s != LRCCS_OK) return s;
    drop_iter_graph(c);
    lrccs_plan best = {};
    double best_ms = time_plan(c, best, n_iter, st);
    if (best_ms < 0.0) {
        restore_state(c, st);
        c->plan = lrccs_plan{};
        set_err(c, "lrccs_autotune: the default plan failed to run");
        return LRCCS_E_CUDA;
    }
    // one field at a time, starting from the defaults
    const int txs[] = {2, 4, 8, 16, 32}, cgs[] = {1, 2, 3, 4, 6, 8}, rgs[] = {1, 2, 4, 8};
    for (int v : txs) {
        if (!fwd_tile_ok(v, c->r, c->nx, c->ny, c->dev_smem_optin)) continue;
        lrccs_plan p = best;
        p.fwd_tx = v;
        const double ms = time_plan(c, p, n_iter, st);
        if (ms >= 0.0 && ms < best_ms) best_ms = ms, best = p;
    }
    for (int v : cgs) {
        if (v > c->nc) continue;
        lrccs_plan p = best;
        p.coil_groups = v;
        const double ms = time_plan(c, p, n_iter, st);
        if (ms >= 0.0 && ms < best_ms) best_ms = ms, best = p;
    }
    if (c->general)
        for (int v : rgs) {
            if (v > c->nc) continue;
            lrccs_plan p = best;
            p.row_groups = v;
            const double ms = time_plan(c, p, n_iter, st);
            if (ms >= 0.0 && ms < best_ms) best_ms = ms, best = p;
        }
    c->plan = best;
    s = restore_state(c, st);
    if (s != LRCCS_OK) return s;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d %d %d\n", key, best.fwd_tx, best.coil_groups, best.row_groups);
            fclose(f);
        }
    }
    if (out) *out = best;
    return LRCCS_OK;
}

// ---------------------------------------------------------------- batched slices

struct lrccs_batch {
    std::vector<lrccs_ctx *> ctxs;
    std::vector<unsigned long long> gens;   // each context's graph generation the batch was built from
    cudaStream_t stream;
    cudaGraphExec_t exec;
    int n_iter;
};

extern "C" lrccs_status lrccs_batch_create(lrccs_ctx *const *ctxs, int32_t count, void *cuda_stream,
                                           lrccs_batch **out) {
    if (!ctxs || count < 1 || !out) {
        set_err(nullptr, "lrccs_batch_create: need contexts and out");
        return LRCCS_E_INVALID;
    }
    *out = nullptr;
    lrccs_batch *b = new (std::nothrow) lrccs_batch();
    if (!b) return LRCCS_E_NOMEM;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) {
            delete b;
            set_err(nullptr, "lrccs_batch_create: null context");
            return LRCCS_E_INVALID;
        }
        b->ctxs.push_back(ctxs[i]);
    }
    b->gens.assign(count, 0);
    b->stream = (cudaStream_t)cuda_stream;
    b->exec = nullptr;
    b->n_iter = 0;
    *out = b;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_batch_iterate(lrccs_batch *b, int32_t n_iter) {
    if (!b || n_iter < 1) {
        set_err(nullptr, "lrccs_batch_iterate: null batch or n_iter < 1");
        return LRCCS_E_INVALID;
    }
    bool rebuild = !b->exec || b->n_iter != n_iter;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        lrccs_ctx *c = b->ctxs[i];
        if (!c->initialized) {
            set_err(nullptr, "lrccs_batch_iterate: context %zu has no data (lrccs_init first)", i);
            return LRCCS_E_STATE;
        }
        if (c->need_h) {
            lrccs_status s = warm_start(c);
            if (s != LRCCS_OK) return s;
        }
        if (!ensure_iter_graph(c, n_iter)) {
            set_err(nullptr, "lrccs_batch_iterate: context %zu cannot capture its iterations (created stream needed)",
                    i);
            return LRCCS_E_CUDA;
        }
        if (b->gens[i] != c->iter_gen) rebuild = true;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            return LRCCS_E_CUDA;
        }
    }
    if (rebuild) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        cudaGraph_t parent = nullptr;
        cudaError_t e = cudaGraphCreate(&parent, 0);
        cudaGraphNode_t prev = nullptr;
        for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i) {
            cudaGraphNode_t node = nullptr;
            e = cudaGraphAddChildGraphNode(&node, parent, prev ? &prev : nullptr, prev ? 1 : 0,
                                           b->ctxs[i]->iter_graph);
            prev = node;
            b->gens[i] = b->ctxs[i]->iter_gen;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, parent, 0);
        if (parent) cudaGraphDestroy(parent);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->exec = nullptr;
            set_err(nullptr, "lrccs_batch_iterate: building the batch graph failed: %s", cudaGetErrorString(e));
            return LRCCS_E_CUDA;
        }
        b->n_iter = n_iter;
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
        cudaGetLastError();
        set_err(nullptr, "lrccs_batch_iterate: graph launch failed");
        return LRCCS_E_CUDA;
    }
    for (lrccs_ctx *c : b->ctxs) {
        for (int k = 0; k < KID_COUNT; ++k) c->launches[k] += c->iter_counts[k];
        c->t += n_iter;
    }
    return LRCCS_OK;
}

extern "C" void lrccs_batch_destroy(lrccs_batch *b) {
    if (!b) return;
    if (b->exec) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->exec);
    }
    delete b;
}

extern "C" lrccs_status lrccs_forward_transform(lrccs_ctx *c, void *d_T, size_t bytes) {
    if (!c || !d_T) return LRCCS_E_INVALID;
    if (!c->initialized || c->need_h) {
        set_err(c, "lrccs_forward_transform: no data and subspace loaded (lrccs_init first)");
        return LRCCS_E_STATE;
    }
    const size_t need = (size_t)c->nc * c->n * c->r * sizeof(float2);
    if (bytes < need) {
        set_err(c, "lrccs_forward_transform: destination holds %zu bytes, %zu needed", bytes, need);
        return LRCCS_E_INVALID;
    }
    CK(launch_forward(c));
    CK(cudaMemcpyAsync(d_T, c->d_T, need, cudaMemcpyDeviceToDevice, c->stream));
    return sync_status(c);
}

extern "C" lrccs_status lrccs_gdqr_phases(lrccs_ctx *c, int32_t enable, double *out) {
    if (!c) return LRCCS_E_INVALID;
    // the stamps of k_gdqr per block: 9 clock64() points, then the global
    // timer (ns) at entry and exit
    const int G = c->gd_grid, NTS = 11, NCLK = 9;
    if (out) {
        if (!c->d_gdts) {
            set_err(c, "lrccs_gdqr_phases: phase timing is off");
            return LRCCS_E_STATE;
        }
        std::vector<long long> h((size_t)G * NTS);
        CK(cudaStreamSynchronize(c->stream));
        CK(cudaMemcpy(h.data(), c->d_gdts, h.size() * sizeof(long long), cudaMemcpyDeviceToHost));
        for (int i = 0; i + 1 < NCLK; ++i) {
            double sum = 0.0, mx = 0.0;
            for (int b = 0; b < G; ++b) {
                const double d = (double)(h[(size_t)b * NTS + i + 1] - h[(size_t)b * NTS + i]);
                sum += d;
                mx = d > mx ? d : mx;
            }
            out[2 * i] = sum / G;
            out[2 * i + 1] = mx;
        }
        long long e0 = h[NCLK], e1 = h[NCLK], x1 = h[NCLK + 1];
        for (int b = 0; b < G; ++b) {
            const long long e = h[(size_t)b * NTS + NCLK], x = h[(size_t)b * NTS + NCLK + 1];
            e0 = e < e0 ? e : e0;
            e1 = e > e1 ? e : e1;
            x1 = x > x1 ? x : x1;
        }
        out[2 * (NCLK - 1)] = (double)(x1 - e0);       // first entry to last exit (ns)
        out[2 * (NCLK - 1) + 1] = (double)(e1 - e0);   // spread of the blocks' entries (ns)
    }
    if (enable && !c->d_gdts) {
        // k_gdqr's stamps, then k_bstep's (the same layout, after them)
        if (!dalloc(c, &c->d_gdts, (size_t)2 * G * NTS)) return LRCCS_E_NOMEM;
        CK(cudaMemset(c->d_gdts, 0, (size_t)2 * G * NTS * sizeof(long long)));
        drop_iter_graph(c);   // captured iterations take the stamps from now on
    } else if (!enable && c->d_gdts && !out) {
        drop_iter_graph(c);
        cudaFree(c->d_gdts);
        c->d_gdts = nullptr;
    }
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_bstep_phases(lrccs_ctx *c, double *out) {
    if (!c || !out) return LRCCS_E_INVALID;
    if (!c->d_gdts) {
        set_err(c, "lrccs_bstep_phases: phase timing is off");
        return LRCCS_E_STATE;
    }
    // k_bstep's global-timer stamps (11 per block, for the blocks b < gd_grid
    // that ran) follow k_gdqr's in the phase-timing buffer
    const int G = c->gd_grid, NTS = 11, NST = 11;
    const int nb = c->n_used < G ? c->n_used : G;
    std::vector<long long> h((size_t)G * NTS);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(h.data(), c->d_gdts + (size_t)G * NTS, h.size() * sizeof(long long), cudaMemcpyDeviceToHost));
    if (nb < 1) return LRCCS_E_STATE;
    for (int i = 0; i + 1 < NST; ++i) {
        double sum = 0.0, mx = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double d = (double)(h[(size_t)b * NST + i + 1] - h[(size_t)b * NST + i]);
            sum += d;
            mx = d > mx ? d : mx;
        }
        out[2 * i] = sum / nb;
        out[2 * i + 1] = mx;
    }
    long long e0 = h[0], e1 = h[0], x1 = h[NST - 1];
    for (int b = 0; b < nb; ++b) {
        const long long e = h[(size_t)b * NST], x = h[(size_t)b * NST + NST - 1];
        e0 = e < e0 ? e : e0;
        e1 = e > e1 ? e : e1;
        x1 = x > x1 ? x : x1;
    }
    out[2 * (NST - 1)] = (double)(x1 - e0);
    out[2 * (NST - 1) + 1] = (double)(e1 - e0);
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_test_wait_timeout(lrccs_ctx *c, int32_t enable) {
    if (!c) return LRCCS_E_INVALID;
    c->test_timeout = enable ? 1 : 0;
    return LRCCS_OK;
}

extern "C" lrccs_status lrccs_synchronize(lrccs_ctx *c) {
    if (!c) return LRCCS_E_INVALID;
    return sync_status(c);
}
