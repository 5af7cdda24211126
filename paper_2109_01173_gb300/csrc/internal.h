// Internal declarations shared by the libmofem translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cublas_v2.h>
#include <atomic>
#include <cstdint>
#include <vector>

#include "../../include/mofem.h"

#define MOFEM_MAX_TERMS 8

// Bit flags written by kernels into the device status word (ctx->d_status).
enum : int {
    DEV_ERR_TIMEOUT = 1,     // a bounded mbarrier wait gave up (tcgen05 GEMM)
    DEV_ERR_NONFINITE = 2,   // NaN/Inf met in a recurrence scalar
    DEV_ERR_BREAKDOWN = 4,   // <Q, L(Q)> <= 0
};

// Per-instance scalar state of the device-resident PCG (FP64).
struct PcgScalars {
    double rz;          // <R, Z> of the current iterate
    double rzo;         // <R_new, Z_old> (flexible beta numerator correction)
    double alpha;       // step of the current iteration
    double beta;        // direction coefficient for the next iteration
    double rr0;         // ||R_0||^2 of this (inner) solve
    double rr;          // ||R||^2 after the last update
    double tol2;        // stop when rr <= tol2
    double rscale;      // scale applied to the FP16 operand copy of R (undone on the GEMM output)
    double alpha_pend;  // mixed form: alpha of the last even iteration, not yet added to the correction
    int iters;          // iterations done in this (inner) solve
    int active;         // 1 while not converged
    int status;         // DEV_ERR_* bits
    int pad;
};

// Fixed partial-sum layout: every reduction writes one double per CTA into a
// slice of `partials`, later summed in a fixed order (deterministic).
struct Partials {
    double* qlq;    // <Q, L(Q)>            [batch][n_apply_ctas]
    double* rr;     // ||R||^2 after update [batch][n_upd_ctas]
    double* rzo;    // <R_new, Z_old>       [batch][n_upd_ctas]
    double* rz;     // <R, Z_new>           [batch][n_rz_ctas]
    double* lqz;    // <L(Q), Z>            [batch][n_apply_ctas] (packed apply: flexible beta without Z_old)
    int n_apply, n_upd, n_rz;
};

struct TcPlan {                 // one tensor-core precision (BF16 or TF32)
    bool ready = false;
    int esize = 0;              // operand bytes (2 bf16, 4 tf32)
    void* Q1 = nullptr;  void* Q1T = nullptr;   // [batch][q][ld] operand copies
    void* Q2 = nullptr;  void* Q2T = nullptr;   // [q][ld] (shared)
    void* Rop = nullptr;                        // GEMM1 A operand (R rounded), [batch][q][ld]
    void* X1T = nullptr; void* WT = nullptr; void* Y = nullptr;  // intermediates
    unsigned* panel_cnt = nullptr;  // GEMM-chain panel counters [3][batch][panels] + end ticket
    int n_panel_cnt = 0;
    CUtensorMap mA[4], mB[4];
    CUtensorMap mO[3];          // TMA-store maps of the intermediates X1T, WT, Y
};

struct mofem_ctx {
    int batch = 1, k = 1, deg = 1, K = 1, P = 3, n = 0, q = 0, nq = 0, NT = 5;
    mofem_bc bc = MOFEM_BC_DIRICHLET;
    mofem_opts opts{};
    int ld = 0;                  // leading dimension of internal q x q matrices (multiple of 64)
    int div_product = 0;         // preconditioner divisor: lambda_a * mu_b (product form) instead of lambda_a + mu_b
    int apply_seg_div = 1;       // operator-apply tile height: rows per CTA of one wave / apply_seg_div (tuned)
    int off = 1;                 // node index of trimmed row 0 (1 Dirichlet, 0 Neumann)
    std::vector<double> gamma;   // per instance
    int dev = 0;

    // banded tables, diagonal-major: tab[term][j][row] = S_term[row][row + j - K]
    double* S64 = nullptr;  float* S32 = nullptr;   // [batch][NT][P][q]
    float* Srow32 = nullptr;   // [batch][q][s_row] FP32 S rows, coefficient t*P + j at t*P + j (packed apply)
    float* Sdf = nullptr;     // plain S tables as double-float: hi plane then lo plane, each [batch][NT][P][q]
    float* Tdf = nullptr;     // plain T tables as double-float: hi plane then lo plane, each [NT][P][q]
    // difference-form tables as double-float (same planes and shapes): off the diagonal slot the
    // plain coefficient, on it the exact row sum of the FP64 coefficients; term 0's t-table holds
    // N = D^{-1}(M_t - D) off the diagonal and D = rowsum M_t on it (exact mass split)
    float* Sdd = nullptr;
    float* Tdd = nullptr;
    float* Srdf = nullptr;    // right-hand-side mass factors as double-float: [hi | lo] of [batch][P][q]
    float* Trdf = nullptr;    // and [hi | lo] of [P][q]
    int s_row = 0;             // floats per Srow32 row
    double* T64 = nullptr;  float* T32 = nullptr;   // [NT][P][q]
    double* Sr64 = nullptr; double* Tr64 = nullptr; // RHS mass factors: [batch][P][q], [P][q] (offset off)
    double* Smf64 = nullptr; double* Tmf64 = nullptr; // untrimmed masses M_s[h], M_t: [batch][P][n], [P][n]
                                                      // (T with its row sum in the diagonal slot)

    // preconditioner eigen data (FP64 masters)
    double* Q1_64 = nullptr;   // [batch][q][ld]  Q1 row-major (columns = eigenvectors)
    double* Q2_64 = nullptr;   // [q][ld]
    double* lam64 = nullptr;   // [batch][ld] (padded with 1)
    double* mu64 = nullptr;    // [ld]
    float* lam32 = nullptr; float* mu32 = nullptr;
    TcPlan tc[3];              // [0] TF32, [1] BF16, [2] FP16

    // FP64-form workspaces (lazily allocated)
    double* w64 = nullptr;     // 8 matrices [batch][q][ld]
    // mixed-form workspaces (lazily allocated)
    float* w32 = nullptr;      // 6 matrices [batch][q][ld]: (spare), R, Z, Q_a, Q_b, L(Q)
    double* U64m = nullptr;    // [batch][q][ld] FP64 iterate of the mixed form
    double* Bm64 = nullptr;    // [batch][q][ld] FP64 right-hand side
    double* R64 = nullptr;     // [batch][q][ld] FP64 true residual
    double* d_part = nullptr;  // partial sums
    Partials part{};
    PcgScalars* d_sc = nullptr;  // [batch]
    int* d_status = nullptr;     // device error bits
    unsigned* d_ctr = nullptr;   // [5][batch] CTA tickets for last-CTA finalisation (zeroed, self-resetting)
    double* d_red = nullptr;     // small scratch for reductions [batch * 8]

    cublasHandle_t cublas = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // captured graphs of one PCG iteration, keyed by precision
    cudaGraphExec_t it_graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t loop_graph[4] = {nullptr, nullptr, nullptr, nullptr};
    int it_graph_max_iter[4] = {0, 0, 0, 0};
    bool host_stepped[4] = {false, false, false, false};   // conditional graph unavailable for this precision
};

// ---- error helpers -------------------------------------------------------
#define MOFEM_CUDA_TRY(x)                                              \
    do {                                                              \
        cudaError_t e_ = (x);                                         \
        if (e_ != cudaSuccess) {                                      \
            mofem_set_last_error(cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? MOFEM_ERR_OOM : MOFEM_ERR_CUDA; \
        }                                                             \
    } while (0)

#define MOFEM_TRY(x)                        \
    do {                                    \
        mofem_status s_ = (x);              \
        if (s_ != MOFEM_OK) return s_;      \
    } while (0)

void mofem_set_last_error(const char* msg, const char* file, int line);

// ---- setup (setup.cpp) ---------------------------------------------------
mofem_status mofem_build(mofem_ctx* c, const mofem_profile* g1, const mofem_profile* g2,
                         const double* gamma, cudaStream_t st);
void mofem_free(mofem_ctx* c);

// ---- kernels (apply.cu) --------------------------------------------------
// Y = L(X) for every instance; optional fused prologue X = Z + beta X_prev and
// partial <X, Y>; see apply.cu for the modes.
enum ApplyMode { APPLY_PLAIN = 0, APPLY_QUPDATE = 1, APPLY_RESIDUAL = 2 };

struct ApplyArgs {
    const void* X; long long x_bs; int x_ld;     // input; Q_prev in QUPDATE mode
    void* Y; long long y_bs; int y_ld;           // output
    const void* Z; void* Xnew;                    // QUPDATE: X := Z + beta X_prev, written to Xnew
    const void* Bm;                               // RESIDUAL: Y = Bm - L(X)
    const void* S; long long s_bs;                // S tables [batch][nt][P][rows_out]
    const void* T;                                // T tables [nt][P][cols_out]
    int rows_in, cols_in, off, rows_out, cols_out;
    double* partial;                              // per-CTA FP64 partials or nullptr
    const PcgScalars* sc;                         // QUPDATE: skip inactive instances, iteration count
    const double* rz_cur; const double* rz_prev; const double* rzo;   // QUPDATE beta sources
    int n_rz, n_rzo, flex;
};
mofem_status launch_apply(int K, int nt, bool fp64, int mode, const ApplyArgs& a, int batch, cudaStream_t st);
int apply_rows_per_cta(int K);

// PCG form of the apply on internal buffers (TMA staging): Q = Z + beta Q_prev
// (written to Qnew), L(Q) -> LQ, partial <Q, L(Q)>, last CTA sets alpha.
struct ApplyPcgArgs {
    const void* S; long long s_bs; const void* T;
    int q, ld; long long bs;
    void* Qnew; void* LQ;
    double* partial; unsigned* counter;
    double* partial2;   // packed FP32 apply: per-CTA <L(Q), Z>, finalised into rzo = rz - alpha <L(Q), Z> (or null)
    PcgScalars* sc; int use_sc;
    int* status;
    int seg_div;   // streaming apply: segments per strip x seg_div (1: one wave of CTAs; 0 reads as 1)
};
mofem_status pcg_direction(mofem_ctx* c, const void* Z, const void* Qp, const double* beta, const double* rz,
                           void* Q, void* LQ, int ld, double* alpha, bool fp64, cudaStream_t st);
// R -= L(d) in double-float arithmetic, d = dh + dl per instance (internal layout),
// and per-CTA FP64 partials of ||R||^2 (nblk per instance).
mofem_status launch_residual_update_df(const mofem_ctx* c, const float* dh, const float* dl, double* R,
                                       double* partial, int* nblk, cudaStream_t st);
int residual_update_df_ctas(int K, int q);   // partials per instance of the above
// The same in difference form with exact row sums and exact input differences (the step
// from U = 0, of the size of U); same grid and partials.  UNSUPPORTED where not served.
mofem_status launch_residual_update_dfd(const mofem_ctx* c, const float* dh, const float* dl, double* R,
                                        double* partial, int* nblk, cudaStream_t st);
bool residual_update_dfd_ok(const mofem_ctx* c);

// One-time launch set-up (function attributes, occupancy queries) is kept per device:
// a process may drive several GPUs, and the heterogeneous-batch runtime launches from
// several host threads.
constexpr int MOFEM_MAX_DEV = 64;
inline int dev_slot() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MOFEM_MAX_DEV) d = 0;
    return d;
}
// Set the kernel's dynamic shared-memory limit once per device.
template <typename F>
inline cudaError_t smem_attr_once(F* kern, int bytes, std::atomic<bool> (&done)[MOFEM_MAX_DEV]) {
    std::atomic<bool>& d = done[dev_slot()];
    if (d.load(std::memory_order_acquire)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) d.store(true, std::memory_order_release);
    return e;
}
// B = M_s F M_t^T (right-hand side; F n x n nodal, ld n, FP64; B q x q, b_ld) in double-float
// arithmetic; MOFEM_ERR_UNSUPPORTED where the tables are missing.
mofem_status launch_rhs_df(const mofem_ctx* c, const double* F, double* B, long long b_bs, int b_ld, cudaStream_t st);
mofem_status launch_apply_pcg(int K, int nt, bool fp64, const CUtensorMap& mZ, const CUtensorMap& mQ,
                              const CUtensorMap* mS,
                              const ApplyPcgArgs& a, int batch, cudaStream_t st);
// Geometry of the PCG-form apply launched for (K, nt, precision): output rows
// per CTA, rows per staging box (TMA map), floats per S row of the streaming apply.
int apply_pcg_rows_per_cta(int K, int nt, bool fp64);
int apply_pcg_box_rows(int K, int nt, bool fp64);
int apply_pcg_s_box_rows();
int apply_pcg_ctas_per_instance(int K, int nt, bool fp64, int q, int batch);
bool apply_pcg_packed(int K, int nt, bool fp64);
int apply_s_row_floats(int K, int nt);
// Coefficient rows of the streaming apply in push form (per input row: the partial sums
// and row sum of each difference term, the matrix column of each plain term) instead of
// the S rows themselves.
bool apply_push_layout();
mofem_status make_row_map(CUtensorMap* m, const void* base, int esize, int cols, int rows, int batch, int ld,
                          int box_cols, int box_rows);

// ---- BLAS-1 / control kernels (blas1.cu) ----------------------------------
mofem_status launch_convert(const void* src, int src_kind, long long s_bs, int s_ld,
                            void* dst, int dst_kind, long long d_bs, int d_ld,
                            int rows, int cols, int batch, cudaStream_t st);   // kinds: 0 f32, 1 f64, 2 bf16, 3 f16
// dst (FP16) = src (FP32) * sc[inst].rscale
mofem_status launch_convert_scaled_f16(const float* src, long long s_bs, int s_ld, void* dst, long long d_bs, int d_ld,
                                       int rows, int cols, int batch, const PcgScalars* sc, cudaStream_t st);
// sc[inst].rscale = sqrt(q*q / sum(partials[inst])) (unit-RMS scale of R)
mofem_status launch_set_rscale(PcgScalars* sc, const double* part, int nper, int batch, double count, cudaStream_t st);
// operand kind of a tensor-core plan: 0 TF32 (f32 storage), 1 BF16, 2 FP16
inline int plan_of(mofem_precision p) { return p == MOFEM_MIXED_BF16 ? 1 : (p == MOFEM_MIXED_FP16 ? 2 : 0); }
inline int conv_kind_of_plan(int which) { return which == 1 ? 2 : (which == 2 ? 3 : 0); }
mofem_status launch_transpose64(const double* src, long long s_bs, double* dst, long long d_bs,
                                int n, int ld, int batch, cudaStream_t st);
mofem_status launch_transpose64_ld(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs,
                                   int d_ld, int n, int batch, cudaStream_t st);
mofem_status launch_hadamard_div64(double* W, long long bs, int ld, int q, const double* lam,
                                   long long lam_bs, const double* mu, int batch, int product, cudaStream_t st);
mofem_status launch_axpy_into64(double* U64, long long u_bs, int u_ld, const float* dU, long long d_bs,
                                int d_ld, int q, int batch, cudaStream_t st);

// ---- tensor-core GEMMs (gemm_tc.cu) ------------------------------------------
// Four GEMMs of the reduced-approach preconditioner on the operand already in
// plan.Rop; writes Z (FP32) and, if rz_partial, the <R, Z> partials (R32 = R in FP32).
mofem_status tc_prepare(mofem_ctx* c, int which, cudaStream_t st);
// z_internal: Z is a library buffer whose row padding may be written (with zeros)
mofem_status tc_precond(const mofem_ctx* c, int which, const float* R32, long long r_bs, int r_ld, float* Z,
                        int z_ld, long long z_bs, double* rz_partial, PcgScalars* sc, cudaStream_t st,
                        bool z_internal = false);
int tc_rz_ctas(const mofem_ctx* c);
mofem_status tc_gemm_one(const mofem_ctx* c, int which, int idx, float* Z, cudaStream_t st);
struct TcBuffers {   // caller-provided BF16 buffers of the preconditioner GEMMs
    void *Q1, *Q1T, *Q2, *Q2T, *Rop, *X1T, *WT, *Y;
    int ld;
};
mofem_status tc_precond_buffers(const mofem_ctx* c, const TcBuffers& b, float* Z, int z_ld, long long z_bs,
                                cudaStream_t st);
mofem_status bench_kernel(mofem_ctx* c, int kernel, mofem_precision prec, int reps, cudaStream_t st);
// Heterogeneous launch: the preconditioner chains of several handles (any q, one operand
// precision) in one persistent launch; descriptors built once in device memory.
struct TcGroupArgs {
    const mofem_ctx* c;
    const float* R32;      // FP32 residual (internal layout) for the fused <R, Z>
    float* Z;              // output (internal layout; row padding may be written)
    double* rz_partial;    // <R, Z> partial slots
};
struct TcMulti {
    void* d_groups = nullptr;      // per-group chain descriptors (device)
    int* d_ubase = nullptr;        // unit bases (device)
    unsigned* d_ctr = nullptr;     // launch counters: end ticket, unit counter, order word
    int ngroups = 0, units = 0, which = 0;
};
mofem_status tc_multi_build(const TcGroupArgs* ga, int n, int which, TcMulti* out);
mofem_status tc_multi_launch(const TcMulti& m, cudaStream_t st);
void tc_multi_free(TcMulti* m);

// ---- solver (solver.cu) ------------------------------------------------------
mofem_status solver_init(mofem_ctx* c, cudaStream_t st);
mofem_status op_apply(mofem_ctx* c, bool fp64, const void* X, long long x_bs, int x_ld, void* Y, long long y_bs,
                      int y_ld, double* partial, cudaStream_t st);
mofem_status op_rhs(mofem_ctx* c, const double* F, double* Bout, long long b_bs, int b_ld, cudaStream_t st);
mofem_status precond64(mofem_ctx* c, const double* R, long long r_bs, int r_ld, double* Z, long long z_bs,
                       int z_ld, cudaStream_t st);
mofem_status precond_tc(mofem_ctx* c, int which, const float* R, long long r_bs, int r_ld, float* Z,
                        long long z_bs, int z_ld, double* rz_partial, PcgScalars* sc, cudaStream_t st);
mofem_status solve_elliptic(mofem_ctx* c, const double* F, double* U, double rtol, int max_iter,
                            mofem_precision prec, mofem_solve_info* info, cudaStream_t st);
mofem_status solve_imex(mofem_ctx* c, double d_u, double tau, const double* Un, const double* Fn, double* Unp1,
                        double rtol, mofem_precision prec, mofem_solve_info* info, cudaStream_t st, double cu = 1.0);
mofem_status dib_run(mofem_ctx* c, const mofem_dib_params& p, double rho, double tau, int n_steps, double* U,
                     double rtol, mofem_precision prec, double* incr, mofem_solve_info* info, cudaStream_t st);
mofem_status dib_equilibrium(const mofem_dib_params& p, double* eta, double* theta);
mofem_status launch_dib_kinetics(const mofem_dib_params& p, double rho, const double* eta, const double* theta,
                                 double* f, double* g, long long n, cudaStream_t st);
mofem_status solve_imex_adjoint(mofem_ctx* c, double d_u, double tau, double r, const double* Lam1, const double* U0,
                                const double* U1, double* Lam0, double* Y, double* dF, double* dd, double* dr, double rtol,
                                mofem_precision prec, mofem_solve_info* info, cudaStream_t st);
mofem_status launch_axpy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld, int rows,
                           int cols, int batch, double a, cudaStream_t st);
void mofem_free_extra(mofem_ctx* c);
// Heterogeneous lockstep solve (solve_fused): graph, branch streams and the multi-group
// GEMM descriptors, kept between solves of the same groups.
struct FusedState {
    TcMulti mc{};
    cudaGraphExec_t loop = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> ev;
    PcgScalars** d_scs = nullptr;
    int* d_bat = nullptr;
    int pe = -1, max_iter = 0, body_kernels = 0;
    bool fixed = false;
};
void fused_free(FusedState* f);
mofem_status set_apply_seg_div(mofem_ctx* c, int div);
// Solve the problems of G handles (one right-hand side and one U per handle, layouts as
// mofem_pcg_solve) in lockstep; mixed forms only (MOFEM_ERR_UNSUPPORTED otherwise, and when
// an FP16 inner solve needs the TF32 retry: the caller then solves the groups apart).
mofem_status solve_fused(mofem_ctx* const* cs, int G, const double* const* F, double* const* U, double rtol,
                         int max_iter, mofem_precision prec, FusedState* f, mofem_solve_info* infos, cudaStream_t st);
