// internal.h -- context layout and kernel launchers of liblrccs (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lrccs.h"

// Indices into the device scalar array ctx->d_scal (float64).
enum {
    SC_GAMMA = 0,   // truncation threshold gamma
    SC_ETA = 1,     // step size
    SC_SD = 2,      // SD(U_{t-1}, U_t) of the last iteration
    SC_GNORM = 3,   // ||grad||_2 of the iteration that set eta
    SC_MBAR = 4,    // mean samples per coil
    SC_ETASET = 5,  // 1 once eta is set
    SC_TCNT = 6,    // iterations run since eta was set (variable step-size schedule)
    SC_COUNT = 8
};

// Indices into the device int array ctx->d_meta.
enum {
    MT_NUSED = 0,   // rows sampled by at least one frame
    MT_NLINES = 1,  // total (frame, line) pairs
    MT_MMIN = 2,    // min_k m_k
    MT_MMAX = 3,    // max_k m_k
    MT_RANK = 4,    // rank chosen by the init
    MT_GENERAL = 5, // 1: some row is only partly sampled (general 2D masks)
    MT_TOTAL = 6,   // sum_k m_k (samples per coil, all frames)
    MT_NU = 7,      // n_u: k-space points sampled by at least one frame (general masks)
    MT_COUNT = 8
};

// Grid-reduction counters.
// CNT_BAR and CNT_BAR + 1: the grid-barrier and exit counters of k_gdqr;
// CNT_BS_BAR and CNT_BS_BAR + 1: those of k_bstep.
enum { CNT_ENERGY = 0, CNT_GRAMX0, CNT_BAR, CNT_BAR_EXIT, CNT_BS_BAR, CNT_BS_EXIT, CNT_COUNT = 8 };

// Kernel ids (launch counting and optional CUDA-event timing).
enum {
    KID_ROWCOUNT = 0, KID_STRUCTURE, KID_FILL_IDX, KID_ENERGY, KID_INIT_ROWS, KID_INIT_COLS, KID_GRAM_X0,
    KID_EIG, KID_U0, KID_GDQR, KID_FWD_COLS, KID_ROW_GRAM, KID_SOLVE, KID_ROW_W, KID_ADJ_COLS,
    KID_IMAGES, KID_CG_INIT, KID_CG_STEP, KID_MEAN_RESID,
    // general (2D) masks
    KID_UNION, KID_FILL_GEN, KID_INIT_GEN, KID_FWD_ROWS, KID_SAMPLE_GRAM, KID_SOLVE_GEN, KID_SAMPLE_W,
    KID_ADJ_ROWS, KID_MEAN_RESID_GEN,
    // model-error correction (Alg. 3) and online tracking (Alg. 5)
    KID_MEC_MASK, KID_MEC_ELEM, KID_MEC_TDFT,
    // precision forms of the forward transform (tcgen05 GEMM)
    KID_TC_A, KID_TC_GEMM, KID_TC_SCALE, KID_TC_B,
    // Z B^H of the gradient; the fused line-mask B-step
    KID_ZB, KID_BSTEP, KID_COUNT
};
extern const char *const kKernelNames[KID_COUNT];

struct prof_rec {
    int kid;
    cudaEvent_t a, b;
    bool graph_owned;   // recorded by nodes of the captured iteration graph
};

struct async_worker;   // host worker thread of the asynchronous tracking calls (api.cu)

struct lrccs_ctx {
    // profiling: launches counted always; kernels in prof_mask timed with events
    long long launches[KID_COUNT];
    long long timed[KID_COUNT];
    double prof_ms[KID_COUNT];
    unsigned long long prof_mask;
    std::vector<prof_rec> pending;
    std::vector<cudaEvent_t> event_pool;

    // the n-iteration loop captured as a CUDA graph on `stream` and replayed by
    // lrccs_iterate; rebuilt when the iteration count, the timed kernels or
    // the shape it was captured for change
    cudaGraphExec_t iter_exec;
    cudaGraph_t iter_graph;             // the captured graph itself (a batch adds it as a child node)
    unsigned long long iter_gen;        // bumped whenever the iteration graph is rebuilt
    long long iter_counts[KID_COUNT];   // kernel launches per replay
    std::vector<prof_rec> iter_prof;    // timing events recorded by the graph
    int iter_n, iter_r, iter_nused, iter_general, iter_nu;
    unsigned long long iter_mask;
    const void *iter_T;
    bool iter_graph_failed;             // capture not possible here: launch directly
    bool capturing;                     // inside the library's own capture
    int capture_iter;                   // iteration being captured
    bool prof_this;                     // the current launch is timed

    lrccs_dims dims;
    lrccs_params prm;
    cudaStream_t stream;
    int ny, nx, n, q, nc, rmax;
    int r;             // rank in use (after init)
    int initialized;   // data and subspace loaded (lrccs_init or a tracking call succeeded)
    int has_u;         // d_U holds a subspace (init, lrccs_set_subspace, lrccs_set_state, tracking)
    int need_h;        // d_U was set from outside: re-orthonormalise it and form U^H Z before iterating
    int t;             // iterations run since init
    int px, py;        // nx / 32, ny / 32
    int nblk;          // blocks of the pixel-parallel init kernels
    int gd_grid;       // blocks of the cooperative GD/QR kernel (all resident)
    int nsm;           // multiprocessors of the device
    int bs_cap[17];    // resident k_bstep<r> blocks for this shape, r = 1..16 (0: rows do not fit)
    int n_used;        // host copy of MT_NUSED
    int n_lines;       // host copy of MT_NLINES
    int m_max;         // host copy of MT_MMAX (largest per-frame sample count per coil)
    int64_t total;     // fp[q] (samples per coil, all frames)
    int general;       // the loaded masks have partly sampled rows: 2D transforms per iteration
    int n_u;           // host copy of MT_NU (general masks)
    size_t gen_cap_q;  // frames the general-mask buffers were allocated for (0: none yet)
    int dev_smem_optin;
    int test_timeout;  // lrccs_test_wait_timeout: the next direct k_gdqr launch waits for an unreachable barrier
    int device;        // CUDA device current at lrccs_create
    size_t create_bytes;   // device bytes allocated by lrccs_create
    async_worker *worker;  // started by the first lrccs_track_minibatch_async
    long long *d_gdts;     // lrccs_gdqr_phases: clock64() stamps of k_gdqr's blocks (NULL: off)
    lrccs_plan plan;       // launch plan of the transform kernels (0 fields: defaults)
    std::string err;

    // geometry / sampling
    float2 *d_twy, *d_twx;       // twiddles w_N^t, N = ny / nx
    float2 *d_smaps;             // nc * n
    int32_t *d_rowcnt;           // q * ny  samples of frame k in row ky
    int32_t *d_rowidx;           // q * ny  line index of row ky in frame k, or -1
    int32_t *d_framerows;        // q * ny  row ky of line i of frame k, at lineptr[k] + i
    int32_t *d_framek;           // q * ny  frame k of frame row lineptr[k] + i
    int32_t *d_mks;              // q       m_k, samples per coil of frame k
    int32_t *d_fpk;              // q + 1   frame sample offsets (the running sum of m_k)
    int32_t *d_rowoff;           // q * ny  first sample of (frame k, row ky) in the frame-ordered sample list
    int32_t *d_lineptr;          // q + 1
    int32_t *d_rfptr;            // ny + 1  frames sampling row ky: rflist[rfptr[ky] .. rfptr[ky+1])
    int32_t *d_rflist;           // q * ny
    int32_t *d_usedrows;         // ny      rows sampled by some frame
    uint8_t *d_rowused;          // ny
    int32_t *d_idx;              // sample indices (capacity q * n)
    int32_t *d_meta;             // MT_COUNT ints, then the eigenvalue order (q ints)
    unsigned int *d_status;      // status word (ST_* bits)
    unsigned int *d_counters;    // CNT_COUNT
    double *d_scal;              // SC_COUNT

    // numerical buffers
    float2 *d_Z;                 // n * q   Z = [A_k^H y_k]   (row-major i*q + k)
    float2 *d_X0;                // n * q   truncated, scaled X0
    float2 *d_T;                 // work: nc * n * rmax (iteration), 2 * nc * fp[q] (init)
    size_t T_cap;                // capacity of d_T in float2
    float2 *d_U;                 // n * rmax  U_t
    float2 *d_Uprev;             // n * rmax  U_{t-1}
    float2 *d_Up;                // n * rmax  gradient, then U+ = U - eta grad
    float2 *d_G;                 // n * rmax  copy of the last gradient (diagnostics)
    float2 *d_B;                 // q * rmax
    float2 *d_P;                 // ny * npairs coil-summed row Grams
    float2 *d_gpart;             // partial sums of the grid reductions (init kernels, k_gdqr)
    size_t gpart_cap;
    double *d_sigma;             // q
    double *d_gram;              // 3 x 2 q q: X0^H X0, A V0, V0^H A V0 (FP64 re, im)
    float2 *d_V;                 // q * q eigenvectors of X0^H X0 (columns)
    float2 *d_Q;                 // q * q rotations of the eigensolver's refine pass
    double2 *d_tot;              // k_gdqr totals: [grad^H grad | U^H grad | U^H U] (iteration), [U+^H U+] (init)
    float2 *d_ZB;                // n * rmax  Z B^H (k_zb)
    float2 *d_hpart;             // gd_grid * q * rmax  per-block partial sums of h = U^H Z (k_gdqr)
    cudaStream_t side;           // parallel branch of the iteration (k_zb beside the adjoint passes)
    cudaEvent_t ev_fork, ev_join;

    // general (2D) masks: the union Omega_u of the frames' samples, kept row by
    // row (points of row ky at u in [uptr[ky], uptr[ky+1]), ascending kx)
    int32_t *d_ucnt;             // n       frames sampling k-space point i
    int32_t *d_uloc;             // n       index of point i among its row's union points, or -1
    int32_t *d_floc;             // n       offset of point i's frame list within its row
    int32_t *d_urow;             // 2 * ny  union points and frame-list entries per row
    int32_t *d_uptr;             // ny + 1
    int32_t *d_ufrow;            // ny + 1
    int32_t *d_upos;             // n       union index of point i, or -1
    int32_t *d_uidx;             // n_u     k-space index of union point u
    int32_t *d_ufptr;            // n_u + 1 frames sampling u: uflist[ufptr[u] .. ufptr[u+1])
    int32_t *d_uflist;           // sum m_k
    int32_t *d_fu;               // sum m_k union index of every frame sample (frame-ordered)
    float2 *d_FU;                // nc * n_u * rmax  F(d_j o U) at the union points (FU[j][u][l])
    float2 *d_Pu;                // n_u * npairs      coil-summed Gram of every union point
    double *d_fpart;             // q * 8 chunks * 2 npairs  per-frame Gram partial sums (FP64)
    uint8_t *d_tflag;            // C sum_k m_k  truncation flags of the init (capacity tflag_cap)
    size_t tflag_cap;

    // model-error correction (Alg. 3): frames in chunks of mec_w = rank_max
    // columns, vectors V[c][i][l] (frame c mec_w + l)
    uint8_t *d_maskc;            // q * n   copy of the loaded masks (per-frame sampling inside N_k)
    float2 *d_mec;               // 5 vectors of mec_nch * n * mec_w: E, S, P, W, and M_prev (MEC-2)
    double *d_mscal;             // gamma, alpha, beta (q each), then reduction partials
    double *d_mout;              // 8 FP64 results of the MEC-2 reductions
    // precision forms: the DFT matrix of the sampled rows as tensor-core
    // operand tiles (bf16 hi / lo, or fp16 in d_tcA0)
    uint16_t *d_tcA0, *d_tcA1;
    uint16_t *d_tcB0, *d_tcB1;   // the B operand d_j o U in the same tiled layout (k_b_operand)
    float *d_tcscale;            // FP16S: [0] max |d| over the coil maps, then max |U| entry per N tile
    float2 *d_twq;               // q twiddles exp(-2 pi i t / q) of the temporal DFT
    int mec_w, mec_nch;
};

void set_err(lrccs_ctx *c, const char *fmt, ...);
void prof_begin(lrccs_ctx *c, int kid);
void prof_end(lrccs_ctx *c, int kid);

// ---- launchers (kernels_*.cu). Each enqueues on c->stream and returns the
// cudaError_t of the launch.
cudaError_t launch_twiddles(float2 *tw, int N, cudaStream_t s);
cudaError_t launch_compact(lrccs_ctx *c, const uint8_t *d_mask, const int64_t *d_fp_user);
cudaError_t launch_fill_lines(lrccs_ctx *c);
// general (2D) masks (kernels_general.cu)
cudaError_t launch_compact_general(lrccs_ctx *c, const uint8_t *d_mask);
cudaError_t launch_init_general(lrccs_ctx *c, const float2 *d_y);   // Z and X0 in one pass (general masks)
cudaError_t launch_iteration_general_front(lrccs_ctx *c);   // forward rows + sample Grams + B-step
cudaError_t launch_iteration_general_back(lrccs_ctx *c);    // W per sample + inverse rows
cudaError_t launch_fwd_rows(lrccs_ctx *c);
cudaError_t launch_fwd_rows_r(lrccs_ctx *c, int r);
cudaError_t launch_adj_rows_r(lrccs_ctx *c, int r);
cudaError_t launch_fwd_cols_on(lrccs_ctx *c, const float2 *src, int r);   // T <- F_y(d_j o src) (n x r src)
cudaError_t launch_adj_cols_to(lrccs_ctx *c, float2 *dst, int r);         // dst <- sum_j conj(d_j) F_y^H T_j
cudaError_t launch_sample_w(lrccs_ctx *c);
cudaError_t launch_adj_rows(lrccs_ctx *c);
cudaError_t launch_mean_resid_general(lrccs_ctx *c, const float2 *d_y, float2 *d_ytil);
// model-error correction and online tracking (kernels_mec.cu)
cudaError_t launch_frame_normal_op(lrccs_ctx *c, const float2 *src, float2 *dst, int w, int k0);
cudaError_t launch_mec_x(lrccs_ctx *c, const float2 *Uprev, const float2 *zbar, float2 *X);
cudaError_t launch_mec_subz(lrccs_ctx *c, const float2 *V);
cudaError_t launch_mec_cg(lrccs_ctx *c, int kind, const float2 *V);
cudaError_t launch_mec_out(lrccs_ctx *c, const float2 *E, const float2 *zbar, float2 *Eout, float2 *Xout);
cudaError_t launch_tdft_fwd(lrccs_ctx *c, const float2 *E, const float2 *S0, const float2 *V, const float2 *Mprev,
                            float2 *M, double *out);
cudaError_t launch_tdft_inv(lrccs_ctx *c, const float2 *M, float omega, float2 *E);
size_t mec_scal_count(int n, int q, int w);
size_t frame_gram_part_count(int q, int rmax);   // doubles of d_fpart
cudaError_t launch_bstep(lrccs_ctx *c);   // B-step only (forward transforms, Grams, solve) at the current U
// precision forms (kernels_tc.cu)
cudaError_t launch_dft_a(lrccs_ctx *c);
cudaError_t launch_forward(lrccs_ctx *c);   // the iteration's forward transform of U (FFT or GEMM)
cudaError_t launch_fwd_gemm(lrccs_ctx *c);
size_t tc_a_elems(int ny);
size_t tc_b_elems(int nc, int ny, int nx, int rmax);
cudaError_t launch_energy(lrccs_ctx *c, const float2 *d_y);
cudaError_t launch_init_adjoint(lrccs_ctx *c, const float2 *d_y);
cudaError_t launch_gram_x0(lrccs_ctx *c);
cudaError_t launch_u0(lrccs_ctx *c);
cudaError_t launch_gdqr(lrccs_ctx *c, int mode);      // F: GD step + Cholesky QR (mode 0: init U+)
cudaError_t launch_zb(lrccs_ctx *c);                  // d_ZB <- Z B^H
cudaError_t launch_solve(lrccs_ctx *c);                // C kernel
bool bstep_fused_ok(const lrccs_ctx *c);               // k_bstep applies (line masks, rows resident)
cudaError_t launch_bstep_fused(lrccs_ctx *c);          // B + C + D in one cooperative launch
int bstep_capacity(int nc, int nx, int q, int r, int smem_optin, int nsm);
cudaError_t launch_iteration(lrccs_ctx *c);            // A .. H for one iteration
cudaError_t launch_images(lrccs_ctx *c, float2 *d_X);
cudaError_t launch_normal_op(lrccs_ctx *c);           // U+ <- A^H A U, rank 1, b_k = 1
cudaError_t launch_fwd_only(lrccs_ctx *c);            // T <- F_y(d_j o U) on the sampled rows
cudaError_t launch_cg_init(lrccs_ctx *c, double *cg);
cudaError_t launch_cg_step(lrccs_ctx *c, double *cg);
cudaError_t launch_mean_resid(lrccs_ctx *c, const float2 *d_y, float2 *d_ytil, int nl_max);
int npairs_of(int r);
bool fwd_tile_ok(int tx, int r, int nx, int ny, int smem_optin);

// Bits of the device status word ctx->d_status.
enum {
    ST_FRAMEPTR_MISMATCH = 1 << 0,
    ST_RESERVED_1 = 1 << 1,   // unused
    ST_NOT_SPD_LS = 1 << 2,
    ST_NOT_SPD_QR = 1 << 3,
    ST_ZERO_SIGMA = 1 << 4,
    ST_TIMEOUT = 1 << 5,
};
