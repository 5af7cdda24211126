// MO-PCG driver (Sec. 5, Eqs. laplace_xnormal_pcg and
// laplace_xnormal_pcg_iteration, standard PCG recurrences; Sec. 6 for the IMEX
// step) on one GPU.
//
// One PCG iteration is a fixed sequence of kernels on device-resident data:
//   apply  : Q = Z + beta Q_prev (fused prologue), L(Q), partial <Q, L(Q)>
//   update : alpha = <R,Z>/<Q,L(Q)>, U += alpha Q, R -= alpha L(Q), partials
//            ||R||^2 and <R_new, Z_old>, BF16 copy of R for the GEMMs
//   control: convergence / breakdown / non-finite tests, sets the graph
//            conditional
//   precond: Z = P^{-1}(R) (four tcgen05 GEMMs, or four DGEMMs in the FP64
//            form), partial <R, Z>
// Two iterations (ping-pong search-direction buffers) form the body of a CUDA
// graph conditional WHILE node, so the whole inner solve runs without host
// round trips.  beta is the flexible (Polak-Ribiere) choice in the mixed form,
// where the rounded preconditioner is not exactly symmetric, and the
// Fletcher-Reeves choice in the FP64 form.
//
// Mixed form: classical iterative refinement: R64 = B - L64(U64) in FP64, an
// inner FP32 solve of L(dU) = R64 to a relative reduction eta, U64 += dU,
// until ||B - L64(U64)||_F <= rtol ||B||_F.
#include "internal.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <algorithm>

mofem_status launch_pcg_update(const mofem_ctx* c, bool fp64, void* U, void* Ulo, void* R, const void* Q,
                               const void* LQ, const void* Zold, void* Rop, int rop_kind, int flex, int max_iter,
                               bool fixed, const cudaGraphConditionalHandle* cond, cudaStream_t st,
                               bool use_scalars = true, const void* Qprev = nullptr, int lazy_phase = -1);
mofem_status launch_fold_df(double* U64, float* hi, float* lo, long long bs, int batch, const PcgScalars* sc,
                            const float* Qpend, int write_d, cudaStream_t st);
mofem_status launch_scale_copy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld,
                                 int rows, int cols, int batch, double scale, cudaStream_t st);
mofem_status launch_pcg_init(const mofem_ctx* c, const double* rr_partials, int n_rr, const double* ref2, double rtol,
                             cudaStream_t st);
mofem_status launch_dot_partials(const void* A, const void* B, bool fp64, long long bs, long long n, int batch,
                                 double* part, int nblk, cudaStream_t st, PcgScalars* sc = nullptr,
                                 unsigned* counter = nullptr, int flex = 0);
mofem_status launch_imex_rhs(const double* Un, const double* Fn, double* Fbar, int n, int q, int off, double gam,
                             double tau, double cu, int batch, cudaStream_t st);

namespace {

constexpr int W32_U = 0, W32_R = 1, W32_Z = 2, W32_QA = 3, W32_QB = 4, W32_LQ = 5, W32_ULO = 6, W32_N = 7;
constexpr int W64_U = 0, W64_R = 1, W64_Z = 2, W64_QA = 3, W64_QB = 4, W64_LQ = 5, W64_T1 = 6, W64_T2 = 7, W64_N = 8;

size_t per(const mofem_ctx* c) { return (size_t)c->q * c->ld; }
float* w32(const mofem_ctx* c, int i) { return c->w32 + per(c) * c->batch * i; }
double* w64(const mofem_ctx* c, int i) { return c->w64 + per(c) * c->batch * i; }

struct Extra {   // per-handle scratch not in the public struct
    double* res_part = nullptr;   // [batch][n_apply] residual partials
    double* bb_part = nullptr;    // [2][batch][n_rz] partials for ||B||^2 and ||U||^2
    double* ref2 = nullptr;       // [batch] reference norm^2 of the stop test
    double* rz_slots[2] = {nullptr, nullptr};
    void* cublas_ws = nullptr;
    cudaStream_t cap = nullptr;
    int n_res = 0;                 // CTAs of the generic apply (residual partials) per instance
    int n_res_alloc = 0;           // residual partials per instance allocated (generic or double-float update)
    bool maps32 = false, maps64 = false;
    CUtensorMap mZ32, mQA32, mQB32, mS32, mZ64, mQA64, mQB64;   // apply staging maps (PCG form)
    PcgScalars* dir_sc = nullptr;  // [batch] scalars of mofem_pcg_direction (apart from the solver's)
    int body_kernels[4] = {0, 0, 0, 0};   // kernel nodes of the captured two-iteration body, per precision
};

}  // namespace

// Extra scratch lives in a side table keyed by handle (keeps mofem_ctx POD-like).  The
// table is shared by all handles, which threads may create, use and destroy
// concurrently: lookups and changes take a lock; an element stays where it is until
// its handle is freed, so the reference returned is used without it.
#include <map>
#include <mutex>
namespace {
std::mutex& extras_lock() {
    static std::mutex m;
    return m;
}
std::map<const mofem_ctx*, Extra>& extras_map() {
    static std::map<const mofem_ctx*, Extra> m;
    return m;
}
struct ExtrasRef {   // extras()[c]: the handle's entry, created on first use
    Extra& operator[](const mofem_ctx* c) const {
        std::lock_guard<std::mutex> g(extras_lock());
        return extras_map()[c];
    }
};
}  // namespace
static ExtrasRef extras() { return ExtrasRef{}; }

static mofem_status ensure_common(mofem_ctx* c, cudaStream_t st) {
    Extra& e = extras()[c];
    if (c->d_part) return MOFEM_OK;
    const int B = c->batch;
    // one partial per CTA of either PCG-form apply (FP32 and FP64 launches differ)
    c->part.n_apply = std::max(apply_pcg_ctas_per_instance(c->K, c->NT, false, c->q, B),
                               apply_pcg_ctas_per_instance(c->K, c->NT, true, c->q, B));
    const int TG = apply_rows_per_cta(c->K);
    e.n_res = ((c->q + 127) / 128) * ((c->q + TG - 1) / TG);
    e.n_res_alloc = std::max(e.n_res, residual_update_df_ctas(c->K, c->q));
    long long nvec = (long long)per(c) / 4;
    c->part.n_upd = (int)std::max(1LL, std::min(296LL, (nvec + 1023) / 1024));
    c->part.n_rz = tc_rz_ctas(c);
    const size_t n_total =
        (size_t)B * (2 * c->part.n_apply + e.n_res_alloc + c->part.n_upd * 2 + c->part.n_rz * 4) + B;
    MOFEM_CUDA_TRY(cudaMalloc(&c->d_part, n_total * sizeof(double)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_part, 0, n_total * sizeof(double), st));
    double* p = c->d_part;
    c->part.qlq = p; p += (size_t)B * c->part.n_apply;
    c->part.lqz = p; p += (size_t)B * c->part.n_apply;
    e.res_part = p; p += (size_t)B * e.n_res_alloc;
    c->part.rr = p; p += (size_t)B * c->part.n_upd;
    c->part.rzo = p; p += (size_t)B * c->part.n_upd;
    e.rz_slots[0] = p; p += (size_t)B * c->part.n_rz;
    e.rz_slots[1] = p; p += (size_t)B * c->part.n_rz;
    e.bb_part = p; p += (size_t)B * c->part.n_rz * 2;   // ||B||^2 and ||U||^2 partials side by side
    e.ref2 = p;
    c->part.rz = e.rz_slots[0];
    MOFEM_CUDA_TRY(cudaMalloc(&c->d_ctr, sizeof(unsigned) * (4 * B + 1)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned) * (4 * B + 1), st));
    MOFEM_CUDA_TRY(cudaMalloc(&c->d_sc, sizeof(PcgScalars) * B));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_sc, 0, sizeof(PcgScalars) * B, st));
    MOFEM_CUDA_TRY(cudaMalloc(&c->d_status, sizeof(int)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
    MOFEM_CUDA_TRY(cudaMalloc(&c->Bm64, per(c) * B * sizeof(double)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->Bm64, 0, per(c) * B * sizeof(double), st));
    MOFEM_CUDA_TRY(cudaMalloc(&c->R64, per(c) * B * sizeof(double)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->R64, 0, per(c) * B * sizeof(double), st));
    MOFEM_CUDA_TRY(cudaStreamCreateWithFlags(&e.cap, cudaStreamNonBlocking));
    MOFEM_CUDA_TRY(cudaEventCreate(&c->ev0));
    MOFEM_CUDA_TRY(cudaEventCreate(&c->ev1));
    return MOFEM_OK;
}

static mofem_status ensure_w32(mofem_ctx* c, cudaStream_t st) {
    if (c->w32) return MOFEM_OK;
    size_t bytes = per(c) * c->batch * W32_N * sizeof(float);
    MOFEM_CUDA_TRY(cudaMalloc(&c->w32, bytes));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->w32, 0, bytes, st));
    MOFEM_CUDA_TRY(cudaMalloc(&c->U64m, per(c) * c->batch * sizeof(double)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->U64m, 0, per(c) * c->batch * sizeof(double), st));
    return MOFEM_OK;
}

static mofem_status ensure_w64(mofem_ctx* c, cudaStream_t st) {
    Extra& e = extras()[c];
    if (c->w64) return MOFEM_OK;
    size_t bytes = per(c) * c->batch * W64_N * sizeof(double);
    MOFEM_CUDA_TRY(cudaMalloc(&c->w64, bytes));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->w64, 0, bytes, st));
    if (!c->cublas) {
        if (cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS) return MOFEM_ERR_CUDA;
        const size_t ws = 32u << 20;
        MOFEM_CUDA_TRY(cudaMalloc(&e.cublas_ws, ws));
        if (cublasSetWorkspace(c->cublas, e.cublas_ws, ws) != CUBLAS_STATUS_SUCCESS) return MOFEM_ERR_CUDA;
        cublasSetMathMode(c->cublas, CUBLAS_DEFAULT_MATH);
    }
    return MOFEM_OK;
}

// TMA maps of the staged apply tiles over the PCG buffers Z, Q_a, Q_b.
static mofem_status ensure_apply_maps(mofem_ctx* c, bool fp64) {
    Extra& e = extras()[c];
    const int WCT = 128 + 8;
    const int HR = apply_pcg_box_rows(c->K, c->NT, fp64);
    if (fp64 && !e.maps64) {
        MOFEM_TRY(make_row_map(&e.mZ64, w64(c, W64_Z), 8, c->q, c->q, c->batch, c->ld, WCT, HR));
        MOFEM_TRY(make_row_map(&e.mQA64, w64(c, W64_QA), 8, c->q, c->q, c->batch, c->ld, WCT, HR));
        MOFEM_TRY(make_row_map(&e.mQB64, w64(c, W64_QB), 8, c->q, c->q, c->batch, c->ld, WCT, HR));
        e.maps64 = true;
    }
    if (!fp64 && !e.maps32) {
        MOFEM_TRY(make_row_map(&e.mZ32, w32(c, W32_Z), 4, c->q, c->q, c->batch, c->ld, WCT, HR));
        MOFEM_TRY(make_row_map(&e.mQA32, w32(c, W32_QA), 4, c->q, c->q, c->batch, c->ld, WCT, HR));
        MOFEM_TRY(make_row_map(&e.mQB32, w32(c, W32_QB), 4, c->q, c->q, c->batch, c->ld, WCT, HR));
        if (apply_pcg_packed(c->K, c->NT, false)) {
            const int w = c->s_row;
            MOFEM_TRY(make_row_map(&e.mS32, c->Srow32, 4, w, c->q, c->batch, w, w, apply_pcg_s_box_rows()));
        }
        e.maps32 = true;
    }
    return MOFEM_OK;
}

void mofem_free_extra(mofem_ctx* c) {
    Extra e;
    {
        std::lock_guard<std::mutex> g(extras_lock());
        auto it = extras_map().find(c);
        if (it == extras_map().end()) return;
        e = it->second;
        extras_map().erase(it);
    }
    cudaFree(e.cublas_ws);
    cudaFree(e.dir_sc);
    if (e.cap) cudaStreamDestroy(e.cap);
}

// ---- single operations ---------------------------------------------------------
static ApplyArgs apply_args_square(const mofem_ctx* c, bool fp64) {
    ApplyArgs a{};
    a.S = fp64 ? (const void*)c->S64 : (const void*)c->S32;
    a.s_bs = (long long)c->NT * c->P * c->q;
    a.T = fp64 ? (const void*)c->T64 : (const void*)c->T32;
    a.rows_in = a.cols_in = a.rows_out = a.cols_out = c->q;
    a.off = 0;
    return a;
}

mofem_status op_apply(mofem_ctx* c, bool fp64, const void* X, long long x_bs, int x_ld, void* Y, long long y_bs,
                      int y_ld, double* partial, cudaStream_t st) {
    ApplyArgs a = apply_args_square(c, fp64);
    a.X = X; a.x_bs = x_bs; a.x_ld = x_ld;
    a.Y = Y; a.y_bs = y_bs; a.y_ld = y_ld;
    a.partial = partial;
    return launch_apply(c->K, c->NT, fp64, APPLY_PLAIN, a, c->batch, st);
}

mofem_status op_rhs(mofem_ctx* c, const double* F, double* Bout, long long b_bs, int b_ld, cudaStream_t st) {
    // double-float evaluation (HBM-bound; the FP64 pipe of this GPU is slow), FP64 otherwise
    const mofem_status sd = launch_rhs_df(c, F, Bout, b_bs, b_ld, st);
    if (sd != MOFEM_ERR_UNSUPPORTED) return sd;
    ApplyArgs a{};
    a.X = F; a.x_bs = (long long)c->n * c->n; a.x_ld = c->n;
    a.Y = Bout; a.y_bs = b_bs; a.y_ld = b_ld;
    a.S = c->Sr64; a.s_bs = (long long)c->P * c->q; a.T = c->Tr64;
    a.rows_in = a.cols_in = c->n;
    a.rows_out = a.cols_out = c->q;
    a.off = c->off;
    return launch_apply(c->K, 1, true, APPLY_PLAIN, a, c->batch, st);
}

// Y = M~ X for q x q unknowns (FP64): the right-hand-side kernel with the mass
// factors' boundary columns dropped (interior indexing, so they meet zeros).
static mofem_status op_mass(mofem_ctx* c, const double* X, long long x_bs, int x_ld, double* Y, long long y_bs, int y_ld,
                            cudaStream_t st) {
    ApplyArgs a{};
    a.X = X; a.x_bs = x_bs; a.x_ld = x_ld;
    a.Y = Y; a.y_bs = y_bs; a.y_ld = y_ld;
    a.S = c->Sr64; a.s_bs = (long long)c->P * c->q; a.T = c->Tr64;
    a.rows_in = a.cols_in = c->q;
    a.rows_out = a.cols_out = c->q;
    a.off = 0;
    return launch_apply(c->K, 1, true, APPLY_PLAIN, a, c->batch, st);
}

static mofem_status op_residual64(mofem_ctx* c, const double* U, long long u_bs, int u_ld, double* R, double* part,
                                  cudaStream_t st) {
    ApplyArgs a = apply_args_square(c, true);
    a.X = U; a.x_bs = u_bs; a.x_ld = u_ld;
    a.Y = R; a.y_bs = (long long)per(c); a.y_ld = c->ld;
    a.Bm = c->Bm64;
    a.partial = part;
    return launch_apply(c->K, c->NT, true, APPLY_RESIDUAL, a, c->batch, st);
}

// FP64 reduced-approach preconditioner through cuBLAS (row-major data viewed as
// column-major transposes): X1 = R Q2, T2 = Q1^T X1, W = T2 ./ (lam + mu), Y = Q1 W, Z = Y Q2^T.
mofem_status precond64(mofem_ctx* c, const double* R, long long r_bs, int r_ld, double* Z, long long z_bs, int z_ld,
                       cudaStream_t st) {
    MOFEM_TRY(ensure_w64(c, st));
    const int q = c->q, ld = c->ld;
    const double one = 1.0, zero = 0.0;
    cublasSetStream(c->cublas, st);
    double* X1 = w64(c, W64_T1);
    double* T2 = w64(c, W64_T2);
    for (int i = 0; i < c->batch; ++i) {
        const double* Ri = R + r_bs * i;
        double* Zi = Z + z_bs * i;
        const double* Q1 = c->Q1_64 + per(c) * i;
        double* x1 = X1 + per(c) * i;
        double* t2 = T2 + per(c) * i;
        cublasStatus_t s1 = cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, q, q, q, &one, c->Q2_64, ld, Ri, r_ld,
                                        &zero, x1, ld);
        cublasStatus_t s2 = cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_T, q, q, q, &one, x1, ld, Q1, ld, &zero, t2, ld);
        if (s1 != CUBLAS_STATUS_SUCCESS || s2 != CUBLAS_STATUS_SUCCESS) return MOFEM_ERR_CUDA;
    }
    MOFEM_TRY(launch_hadamard_div64(T2, per(c), ld, q, c->lam64, ld, c->mu64, c->batch, c->div_product, st));
    for (int i = 0; i < c->batch; ++i) {
        double* Zi = Z + z_bs * i;
        const double* Q1 = c->Q1_64 + per(c) * i;
        double* x1 = X1 + per(c) * i;   // reuse as Y
        double* t2 = T2 + per(c) * i;
        cublasStatus_t s3 = cublasDgemm(c->cublas, CUBLAS_OP_N, CUBLAS_OP_N, q, q, q, &one, t2, ld, Q1, ld, &zero, x1, ld);
        cublasStatus_t s4 = cublasDgemm(c->cublas, CUBLAS_OP_T, CUBLAS_OP_N, q, q, q, &one, c->Q2_64, ld, x1, ld, &zero,
                                        Zi, z_ld);
        if (s3 != CUBLAS_STATUS_SUCCESS || s4 != CUBLAS_STATUS_SUCCESS) return MOFEM_ERR_CUDA;
    }
    return MOFEM_OK;
}

// Tensor-core preconditioner on a user (or internal) FP32 matrix R.
mofem_status precond_tc(mofem_ctx* c, int which, const float* R, long long r_bs, int r_ld, float* Z, long long z_bs,
                        int z_ld, double* rz_partial, PcgScalars* sc, cudaStream_t st) {
    MOFEM_TRY(tc_prepare(c, which, st));
    TcPlan& p = c->tc[which];
    const long long bs = (long long)per(c);
    if (which == 2) {
        // FP16 operands: R scaled to unit RMS per instance (scale in the scalar state)
        MOFEM_TRY(ensure_w32(c, st));
        float* Rt = w32(c, W32_LQ);   // scratch FP32 copy with zero padding
        MOFEM_TRY(launch_convert(R, 0, r_bs, r_ld, Rt, 0, bs, c->ld, c->q, c->q, c->batch, st));
        MOFEM_TRY(launch_dot_partials(Rt, Rt, false, bs, bs, c->batch, c->part.rr, c->part.n_upd, st));
        MOFEM_TRY(launch_set_rscale(c->d_sc, c->part.rr, c->part.n_upd, c->batch, (double)c->q * c->q, st));
        MOFEM_TRY(launch_convert_scaled_f16(Rt, bs, c->ld, p.Rop, bs, c->ld, c->q, c->q, c->batch, c->d_sc, st));
    } else {
        MOFEM_TRY(launch_convert(R, 0, r_bs, r_ld, p.Rop, conv_kind_of_plan(which), bs, c->ld, c->q, c->q, c->batch,
                                 st));
    }
    return tc_precond(c, which, R, r_bs, r_ld, Z, z_ld, z_bs, rz_partial, sc, st);
}

// ---- PCG iteration (captured) -----------------------------------------------------
static mofem_status pcg_iteration(mofem_ctx* c, mofem_precision prec, int s, int max_iter, bool fixed,
                                  const cudaGraphConditionalHandle* cond, cudaStream_t st, bool with_precond = true) {
    Extra& e = extras()[c];
    const bool fp64 = prec == MOFEM_FP64;
    const int which = plan_of(prec);
    const long long bs = (long long)per(c);
    void *U, *Ulo = nullptr, *R, *Z, *Qn, *Qp, *LQ;
    const CUtensorMap *mZ, *mQp;
    if (fp64) {
        U = w64(c, W64_U); R = w64(c, W64_R); Z = w64(c, W64_Z);
        Qn = w64(c, s % 2 ? W64_QB : W64_QA); Qp = w64(c, s % 2 ? W64_QA : W64_QB); LQ = w64(c, W64_LQ);
        mZ = &e.mZ64; mQp = s % 2 ? &e.mQA64 : &e.mQB64;
    } else {
        U = w32(c, W32_U); Ulo = w32(c, W32_ULO); R = w32(c, W32_R); Z = w32(c, W32_Z);
        Qn = w32(c, s % 2 ? W32_QB : W32_QA); Qp = w32(c, s % 2 ? W32_QA : W32_QB); LQ = w32(c, W32_LQ);
        mZ = &e.mZ32; mQp = s % 2 ? &e.mQA32 : &e.mQB32;
    }
    // 1) Q = Z + beta Q_prev ; LQ = L(Q) ; alpha = <R,Z>/<Q,LQ> (last CTA)
    ApplyPcgArgs a{};
    a.S = fp64 ? (const void*)c->S64 : (const void*)c->S32;
    a.s_bs = (long long)c->NT * c->P * c->q;
    a.T = fp64 ? (const void*)c->T64 : (const void*)c->T32;
    a.q = c->q; a.ld = c->ld; a.bs = bs;
    a.Qnew = Qn; a.LQ = LQ;
    a.partial = c->part.qlq; a.counter = c->d_ctr;
    // the packed FP32 apply also forms <R_new, Z> for the flexible beta (no Z re-read in the update)
    const bool packed = apply_pcg_packed(c->K, c->NT, fp64);
    a.partial2 = packed ? c->part.lqz : nullptr;
    a.sc = c->d_sc; a.use_sc = 1;
    a.status = c->d_status;
    a.seg_div = c->apply_seg_div;
    MOFEM_TRY(launch_apply_pcg(c->K, c->NT, fp64, *mZ, *mQp, fp64 ? nullptr : &e.mS32, a, c->batch, st));
    // 2) R -= alpha LQ ; U += alpha Q (mixed: lazily, two iterations at a time) ; convergence
    //    (last CTA) ; graph condition
    MOFEM_TRY(launch_pcg_update(c, fp64, U, Ulo, R, Qn, LQ, Z, fp64 ? nullptr : c->tc[which].Rop,
                                fp64 ? 0 : (which == 1 ? 1 : (which == 2 ? 2 : 0)), (fp64 || packed) ? 0 : 1,
                                max_iter, fixed, cond, st, true, fp64 ? nullptr : Qp, fp64 ? -1 : (s & 1)));
    // 3) Z = P^{-1}(R) ; rz and beta (last CTA)
    if (!with_precond) {   // heterogeneous lockstep: one GEMM launch for every group (solve_fused)
        if (!fp64 && which == 0)
            MOFEM_TRY(launch_convert(R, 0, bs, c->ld, c->tc[0].Rop, 0, bs, c->ld, c->q, c->q, c->batch, st));
        return MOFEM_OK;
    }
    if (fp64) {
        MOFEM_TRY(precond64(c, (const double*)R, bs, c->ld, (double*)Z, bs, c->ld, st));
        MOFEM_TRY(launch_dot_partials(R, Z, true, bs, bs, c->batch, e.rz_slots[0], c->part.n_rz, st, c->d_sc,
                                      c->d_ctr + 2 * c->batch, 0));
    } else {
        if (which == 0)   // TF32 GEMMs read their own FP32 operand copy of R
            MOFEM_TRY(launch_convert(R, 0, bs, c->ld, c->tc[0].Rop, 0, bs, c->ld, c->q, c->q, c->batch, st));
        MOFEM_TRY(tc_precond(c, which, (const float*)R, bs, c->ld, (float*)Z, c->ld, bs, e.rz_slots[0], c->d_sc, st,
                             true));
    }
    return MOFEM_OK;
}

// Kernel nodes of a captured graph (its memset nodes not counted).
static int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> v(n);
    if (n && cudaGraphGetNodes(g, v.data(), &n) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Build (once per precision) the graph: WHILE(cond) { iteration(0); iteration(1) }.
static mofem_status build_loop_graph(mofem_ctx* c, mofem_precision prec, int max_iter, bool fixed) {
    Extra& e = extras()[c];
    const int pi = (int)prec;
    if (c->loop_graph[pi] && c->it_graph_max_iter[pi] == (fixed ? -max_iter : max_iter)) return MOFEM_OK;
    if (c->loop_graph[pi]) {
        cudaGraphExecDestroy(c->loop_graph[pi]);
        c->loop_graph[pi] = nullptr;
    }
    cudaGraph_t g;
    MOFEM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    MOFEM_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    MOFEM_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MOFEM_CUDA_TRY(cudaStreamBeginCaptureToGraph(e.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    mofem_status s0 = pcg_iteration(c, prec, 0, max_iter, fixed, &h, e.cap);
    mofem_status s1 = s0 == MOFEM_OK ? pcg_iteration(c, prec, 1, max_iter, fixed, &h, e.cap) : s0;
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e.cap, &out);
    if (s1 != MOFEM_OK) {
        cudaGraphDestroy(g);
        return s1;
    }
    MOFEM_CUDA_TRY(ce);
    e.body_kernels[pi] = count_kernel_nodes(body);
    cudaGraphExec_t ex;
    MOFEM_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    c->loop_graph[pi] = ex;
    c->it_graph_max_iter[pi] = fixed ? -max_iter : max_iter;
    return MOFEM_OK;
}

// Host-driven alternative (MOFEM_FLAG_HOST_LOOP): one graph of two iterations
// launched until every instance is inactive.
static mofem_status build_step_graph(mofem_ctx* c, mofem_precision prec, int max_iter, bool fixed) {
    Extra& e = extras()[c];
    const int pi = (int)prec;
    if (c->it_graph[pi] && c->it_graph_max_iter[pi] == (fixed ? -max_iter : max_iter)) return MOFEM_OK;
    if (c->it_graph[pi]) {
        cudaGraphExecDestroy(c->it_graph[pi]);
        c->it_graph[pi] = nullptr;
    }
    MOFEM_CUDA_TRY(cudaStreamBeginCapture(e.cap, cudaStreamCaptureModeRelaxed));
    mofem_status s0 = pcg_iteration(c, prec, 0, max_iter, fixed, nullptr, e.cap);
    mofem_status s1 = s0 == MOFEM_OK ? pcg_iteration(c, prec, 1, max_iter, fixed, nullptr, e.cap) : s0;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e.cap, &g);
    if (s1 != MOFEM_OK) {
        if (g) cudaGraphDestroy(g);
        return s1;
    }
    MOFEM_CUDA_TRY(ce);
    e.body_kernels[pi] = count_kernel_nodes(g);
    cudaGraphExec_t ex;
    MOFEM_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    c->it_graph[pi] = ex;
    c->it_graph_max_iter[pi] = fixed ? -max_iter : max_iter;
    return MOFEM_OK;
}

static mofem_status read_scalars(mofem_ctx* c, std::vector<PcgScalars>& sc, cudaStream_t st) {
    sc.resize(c->batch);
    MOFEM_CUDA_TRY(cudaMemcpyAsync(sc.data(), c->d_sc, sizeof(PcgScalars) * c->batch, cudaMemcpyDeviceToHost, st));
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    return MOFEM_OK;
}

// Fixed-order host sum of per-instance partials (deterministic).
static mofem_status sum_partials(const double* d, int nper, int batch, std::vector<double>& out, cudaStream_t st) {
    std::vector<double> h((size_t)nper * batch);
    MOFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    out.assign(batch, 0.0);
    for (int i = 0; i < batch; ++i)
        for (int j = 0; j < nper; ++j) out[i] += h[(size_t)i * nper + j];
    return MOFEM_OK;
}

// Run one inner solve: R (working precision) holds the start residual, U = 0 or a
// guess already in the U buffer.  Stops at ||R|| <= rtol * sqrt(ref2) (ref2 = ||R0||^2 when null).
static mofem_status run_inner(mofem_ctx* c, mofem_precision prec, int max_iter, bool fixed, const double* ref2_dev,
                              double rtol, cudaStream_t st) {
    Extra& e = extras()[c];
    const bool fp64 = prec == MOFEM_FP64;
    const int which = plan_of(prec);
    const long long bs = (long long)per(c);
    void* R = fp64 ? (void*)w64(c, W64_R) : (void*)w32(c, W32_R);
    void* Z = fp64 ? (void*)w64(c, W64_Z) : (void*)w32(c, W32_Z);
    void* Qp = fp64 ? (void*)w64(c, W64_QB) : (void*)w32(c, W32_QB);
    const size_t esz = fp64 ? 8 : 4;
    MOFEM_TRY(ensure_apply_maps(c, fp64));
    MOFEM_CUDA_TRY(cudaMemsetAsync(Qp, 0, bs * c->batch * esz, st));
    // ||R0||^2 -> init (active flags, tolerance, counters)
    MOFEM_TRY(launch_dot_partials(R, R, fp64, bs, bs, c->batch, c->part.rr, c->part.n_upd, st));
    MOFEM_TRY(launch_pcg_init(c, c->part.rr, c->part.n_upd, ref2_dev, rtol, st));
    // Z0 = P^{-1}(R0) and rz = <R0, Z0> (last-CTA finalisation)
    if (fp64) {
        MOFEM_TRY(precond64(c, (const double*)R, bs, c->ld, (double*)Z, bs, c->ld, st));
        MOFEM_TRY(launch_dot_partials(R, Z, true, bs, bs, c->batch, e.rz_slots[0], c->part.n_rz, st, c->d_sc,
                                      c->d_ctr + 2 * c->batch, 0));
    } else {
        MOFEM_TRY(tc_prepare(c, which, st));
        if (which == 2)   // scale from ||R0|| set by the init kernel
            MOFEM_TRY(launch_convert_scaled_f16((const float*)R, bs, c->ld, c->tc[2].Rop, bs, c->ld, c->q, c->q,
                                                c->batch, c->d_sc, st));
        else
            MOFEM_TRY(launch_convert(R, 0, bs, c->ld, c->tc[which].Rop, conv_kind_of_plan(which), bs, c->ld, c->q,
                                     c->q, c->batch, st));
        MOFEM_TRY(tc_precond(c, which, (const float*)R, bs, c->ld, (float*)Z, c->ld, bs, e.rz_slots[0], c->d_sc, st,
                             true));
    }
    const int pi = (int)prec;
    bool stepped = (c->opts.flags & MOFEM_FLAG_HOST_LOOP) || c->host_stepped[pi];
    if (!stepped) {
        mofem_status gs = build_loop_graph(c, prec, max_iter, fixed);
        if (gs == MOFEM_OK) {
            MOFEM_CUDA_TRY(cudaGraphLaunch(c->loop_graph[pi], st));
            return MOFEM_OK;
        }
        // A device-side loop cannot be built for this precision (cuBLAS kernels in
        // the body of a conditional node are rejected at some sizes): step the
        // two-iteration graph from the host instead, for this and later solves.
        cudaGetLastError();
        c->host_stepped[pi] = true;
    }
    MOFEM_TRY(build_step_graph(c, prec, max_iter, fixed));
    std::vector<PcgScalars> sc;
    for (int guard = 0; guard < max_iter + 2; guard += 2) {
        MOFEM_CUDA_TRY(cudaGraphLaunch(c->it_graph[pi], st));
        MOFEM_TRY(read_scalars(c, sc, st));
        bool any = false;
        for (auto& s : sc) any = any || s.active;
        if (!any) break;
    }
    return MOFEM_OK;
}

static mofem_status finish_info(mofem_ctx* c, mofem_solve_info* info, mofem_status st_code, int iters, int outer,
                                double rel, float ms, long long launches) {
    if (info) {
        info->kernel_launches = launches;
        info->status = st_code;
        info->iterations = iters;
        info->outer_steps = outer;
        info->batch = c->batch;
        info->rel_residual = rel;
        info->ms_total = ms;
    }
    return st_code;
}

// Core solve on Bm64 (already formed).  U: q x q per instance, ld u_ld, FP64,
// in/out.  Stop: ||B - L(U)|| <= rtol * ref, ref = ||B|| (ref_is_r0 = 0) or the
// initial residual norm (ref_is_r0 = 1, IMEX rule).
static mofem_status solve_core(mofem_ctx* c, double* U, long long u_bs, int u_ld, double rtol, int max_iter,
                               mofem_precision prec, int ref_is_r0, mofem_solve_info* info, cudaStream_t st) {
    Extra& e = extras()[c];
    const int B = c->batch, q = c->q, ld = c->ld;
    const long long bs = (long long)per(c);
    const bool fixed = (c->opts.flags & MOFEM_FLAG_FIXED_ITERS) != 0;
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
    MOFEM_CUDA_TRY(cudaEventRecord(c->ev0, st));
    // reference norm ||B||^2 and ||U||^2 (a zero initial guess needs no FP64 apply: R0 = B),
    // both read back with one synchronisation
    std::vector<double> bb, rr, uu, both;
    MOFEM_TRY(launch_dot_partials(c->Bm64, c->Bm64, true, bs, bs, B, e.bb_part, c->part.n_rz, st));
    MOFEM_TRY(launch_dot_partials(U, U, true, u_bs, (long long)q * q, B, e.bb_part + (size_t)B * c->part.n_rz,
                                  c->part.n_rz, st));
    MOFEM_TRY(sum_partials(e.bb_part, c->part.n_rz, 2 * B, both, st));
    bb.assign(both.begin(), both.begin() + B);
    uu.assign(both.begin() + B, both.end());
    bool zero_guess = true;
    for (int i = 0; i < B; ++i) zero_guess = zero_guess && uu[i] == 0.0;
    if (zero_guess) {
        MOFEM_CUDA_TRY(cudaMemcpyAsync(c->R64, c->Bm64, sizeof(double) * bs * B, cudaMemcpyDeviceToDevice, st));
        rr = bb;
    } else {
        MOFEM_TRY(op_residual64(c, U, u_bs, u_ld, c->R64, e.res_part, st));
        MOFEM_TRY(sum_partials(e.res_part, e.n_res, B, rr, st));
    }
    const bool trace = getenv("MOFEM_TRACE") != nullptr;
    std::vector<double> ref2(B);
    for (int i = 0; i < B; ++i) ref2[i] = ref_is_r0 ? rr[i] : bb[i];
    int total_it = 0, outer = 0;
    // ||B||^2 and ||U||^2 dots, the FP64 residual of a nonzero guess, the copy of U into
    // the iterate's layout (the right-hand side is counted by the caller)
    long long launches = 2 + (zero_guess ? 0 : 1) + 1;
    // kernels per inner solve: init sequence (dot, init, then the first preconditioner:
    // operand conversion + GEMM chain, or Hadamard division + dot) + WHILE bodies of two
    // iterations.  libmofem kernels only: a mixed body is counted from its captured graph
    // (apply, update, [TF32 operand copy,] GEMM chain per iteration); the FP64 body's
    // DGEMMs are cuBLAS kernels, so its count is apply, update, division, dot.
    auto inner_launches = [&](int it, mofem_precision pr) -> long long {
        const bool fp64 = pr == MOFEM_FP64;
        const int pb = extras()[c].body_kernels[(int)pr];
        const long long per_body = fp64 ? 2 * 4 : (pb > 0 ? pb : 2 * (pr == MOFEM_MIXED_TF32 ? 4 : 3));
        const long long bodies = std::max(1, (it + 1) / 2);
        return 4 + bodies * per_body;
    };
    mofem_status code = MOFEM_OK;
    std::vector<PcgScalars> sc;
    auto rel_max = [&](const std::vector<double>& r) {
        double m = 0.0;
        for (int i = 0; i < B; ++i) {
            double v;
            if (!std::isfinite(ref2[i]) || !std::isfinite(r[i])) v = NAN;
            else v = ref2[i] > 0 ? std::sqrt(r[i] / ref2[i]) : (r[i] > 0 ? INFINITY : 0.0);
            if (!(v <= m)) m = v;   // NaN propagates
        }
        return m;
    };
    double rel = rel_max(rr);
    // Refinement stalls once the FP64 residual is at its evaluation floor (a step that
    // no longer halves the true residual).  Relative to ||R_0|| (IMEX rule) the step is
    // then as accurate as FP64 can tell and counts as converged; relative to ||B|| it is
    // reported as not converged.
    bool stalled = false;
    auto stall_check = [&](double prev) {
        if (outer >= 1 && std::isfinite(rel) && rel > 0.5 * prev) stalled = true;
    };
    if (prec == MOFEM_FP64) {
        // FP64 MO-PCG from U with stop ||R|| <= rtol ||B|| on the recursively
        // updated residual; if the recomputed true residual misses the target,
        // restart from the current U with the true residual (residual replacement).
        MOFEM_TRY(ensure_w64(c, st));
        const int max_outer = c->opts.max_outer > 0 ? c->opts.max_outer : 20;
        MOFEM_TRY(launch_convert(U, 1, u_bs, u_ld, w64(c, W64_U), 1, bs, ld, q, q, B, st));
        MOFEM_CUDA_TRY(cudaMemcpyAsync(e.ref2, ref2.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
        while (!(rel <= rtol) && outer < max_outer && std::isfinite(rel) && !stalled) {
            const double rel_prev = rel;
            MOFEM_CUDA_TRY(cudaMemcpyAsync(w64(c, W64_R), c->R64, sizeof(double) * bs * B, cudaMemcpyDeviceToDevice, st));
            MOFEM_TRY(run_inner(c, prec, max_iter, fixed, e.ref2, rtol, st));
            MOFEM_TRY(read_scalars(c, sc, st));
            int it = 0;
            for (auto& s : sc) it = std::max(it, s.iters);
            total_it += it;
            ++outer;
            launches += inner_launches(it, MOFEM_FP64) + 2;
            MOFEM_TRY(launch_convert(w64(c, W64_U), 1, bs, ld, U, 1, u_bs, u_ld, q, q, B, st));
            MOFEM_TRY(op_residual64(c, U, u_bs, u_ld, c->R64, e.res_part, st));
            MOFEM_TRY(sum_partials(e.res_part, e.n_res, B, rr, st));
            rel = rel_max(rr);
            stall_check(rel_prev);
            if (trace) fprintf(stderr, "[mofem] fp64 pass %d: iterations %d, rel residual %.3e\n", outer, it, rel);
            if (fixed) break;
        }
    } else {
        MOFEM_TRY(ensure_w32(c, st));
        // effective inner precision: FP16 may fall back to TF32; the product preconditioner's
        // divisor lambda_a mu_b spans ~12 decades, beyond FP16 operand range, so it uses TF32
        mofem_precision pe = (prec == MOFEM_MIXED_FP16 && c->div_product) ? MOFEM_MIXED_TF32 : prec;
        MOFEM_TRY(tc_prepare(c, plan_of(pe), st));
        const int max_outer = c->opts.max_outer > 0 ? c->opts.max_outer : 20;
        // Inner reductions: eta0 for the first step (from zero the FP32 correction
        // equation levels off near 1e-5 of ||B|| at P2, N = 2049); later steps aim
        // straight at rtol, no deeper than eta0 / 10.  Two FP64 residuals instead of
        // three for rtol = 1e-10 on that workload.
        const double eta0 = c->opts.inner_rtol > 0 ? c->opts.inner_rtol : 1e-5;
        // The residual updates track B - L(U) of the FP64 iterate up to their double-float
        // evaluation errors: ~2^-48 q of ||B|| for the step from zero (difference form,
        // 1e-12 at q = 2047), ~1e-13 for a later correction of 1e-5 ||U||; where the
        // difference form is not served, the anchor is an FP64 recomputation.  An FP64
        // evaluation (the t-pass mass product rounded to FP64, then second-differenced)
        // carries ~u q^2 / pi^2 of ||B||, 4.7e-11 at q = 2047: targets below twice that
        // level (or 1e-11) are beyond what an FP64 check of the result could confirm, so
        // such targets, and the MOFEM_FLAG_TRUE_RESIDUAL flag, recompute B - L(U) in FP64
        // after every step, where a stall is the verdict that check would give.
        const double floor_est = std::max(1e-11, 2.0 * 0x1p-53 * (double)q * q / (M_PI * M_PI));
        bool df_update = (c->opts.flags & MOFEM_FLAG_TRUE_RESIDUAL) == 0;
        for (int i = 0; i < B; ++i) df_update = df_update && rtol * rtol * ref2[i] >= floor_est * floor_est * bb[i];
        // the FP64 iterate lives in U64m (internal layout) during the solve
        MOFEM_TRY(launch_convert(U, 1, u_bs, u_ld, c->U64m, 1, bs, ld, q, q, B, st));
        while (!(rel <= rtol) && outer < max_outer && std::isfinite(rel) && !stalled) {
            const double rel_prev = rel;
            // inner tolerance: no further than needed for this step
            double eta = std::max(outer == 0 ? eta0 : 0.1 * eta0, 0.3 * rtol / rel);
            if (eta >= 1.0) eta = 0.5;
            // R32 <- R64 ; converged instances get R = 0 (inactive)
            MOFEM_TRY(launch_convert(c->R64, 1, bs, ld, w32(c, W32_R), 0, bs, ld, q, q, B, st));
            for (int i = 0; i < B; ++i) {
                double ri = ref2[i] > 0 ? std::sqrt(rr[i] / ref2[i]) : 0.0;
                if (ri <= rtol) MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_R) + bs * i, 0, sizeof(float) * bs, st));
            }
            // inner FP32 MO-PCG on the correction (double-float accumulator, zero at
            // start), folded into the FP64 iterate U64m at the end
            MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_U), 0, sizeof(float) * bs * B, st));
            MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_ULO), 0, sizeof(float) * bs * B, st));
            MOFEM_TRY(run_inner(c, pe, max_iter, fixed, nullptr, eta, st));
            MOFEM_TRY(read_scalars(c, sc, st));
            bool bad = false;
            for (auto& s : sc) bad = bad || (s.status & DEV_ERR_NONFINITE) || !std::isfinite(s.rr);
            if (bad && pe == MOFEM_MIXED_FP16) {
                // FP16 operand range exceeded: redo this step with TF32 operands
                if (trace) fprintf(stderr, "[mofem] FP16 inner solve non-finite; repeating the step in TF32\n");
                int it_bad = 0;
                for (auto& s : sc) it_bad = std::max(it_bad, s.iters);
                launches += inner_launches(it_bad, pe) + 1;   // + convert R
                pe = MOFEM_MIXED_TF32;
                MOFEM_TRY(tc_prepare(c, plan_of(pe), st));
                continue;
            }
            // R after this step, updated R -= L(d - err) in double-float arithmetic, err the
            // fold's rounding of U + d (the fold leaves d - err in the correction pair).  A step
            // from zero (d of the size of U; R cancels to ~1e-5 of B) takes the difference form
            // with exact row sums and differences, the iterate set to the pair itself; where
            // that form is not served, R is recomputed in FP64.
            const bool from_zero = outer == 0 && zero_guess;
            const bool upd = df_update && (!from_zero || residual_update_dfd_ok(c));
            const int dmode = !upd ? 0 : (from_zero ? 2 : 1);
            // even iterations leave alpha Q_a pending (lazy correction): the fold adds it
            MOFEM_TRY(launch_fold_df(c->U64m, w32(c, W32_U), w32(c, W32_ULO), bs, B, c->d_sc, w32(c, W32_QA), dmode, st));
            int it = 0;
            for (auto& s : sc) it = std::max(it, s.iters);
            total_it += it;
            ++outer;
            launches += inner_launches(it, pe) + 3;   // + convert R, fold, residual
            int nblk = 0;
            mofem_status du = MOFEM_ERR_UNSUPPORTED;
            if (upd)
                du = from_zero ? launch_residual_update_dfd(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, e.res_part, &nblk, st)
                               : launch_residual_update_df(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, e.res_part, &nblk, st);
            if (du == MOFEM_OK) {
                MOFEM_TRY(sum_partials(e.res_part, nblk, B, rr, st));
            } else {
                if (du != MOFEM_ERR_UNSUPPORTED) return du;
                MOFEM_TRY(op_residual64(c, c->U64m, bs, ld, c->R64, e.res_part, st));
                MOFEM_TRY(sum_partials(e.res_part, e.n_res, B, rr, st));
            }
            rel = rel_max(rr);
            stall_check(rel_prev);
            if (trace)
                fprintf(stderr, "[mofem] outer %d: inner iterations %d (eta %.2e), rel residual %.3e\n", outer, it, eta,
                        rel);
            if (fixed) break;
        }
        MOFEM_TRY(launch_convert(c->U64m, 1, bs, ld, U, 1, u_bs, u_ld, q, q, B, st));
    }
    MOFEM_CUDA_TRY(cudaEventRecord(c->ev1, st));
    // status word and scalar state, read back with one synchronisation
    int dev_status = 0;
    sc.resize(B);
    MOFEM_CUDA_TRY(cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MOFEM_CUDA_TRY(cudaMemcpyAsync(sc.data(), c->d_sc, sizeof(PcgScalars) * B, cudaMemcpyDeviceToHost, st));
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    int sc_status = 0;
    for (auto& s : sc) sc_status |= s.status;
    dev_status |= sc_status;
    if (dev_status & DEV_ERR_TIMEOUT) code = MOFEM_ERR_TIMEOUT;
    else if ((dev_status & DEV_ERR_NONFINITE) || !std::isfinite(rel)) code = MOFEM_ERR_NONFINITE;
    else if (dev_status & DEV_ERR_BREAKDOWN && !(rel <= rtol)) code = MOFEM_ERR_BREAKDOWN;
    else if (!(rel <= rtol) && !fixed && !(stalled && ref_is_r0)) code = MOFEM_ERR_NOT_CONVERGED;
    // + the mixed forms' copy of the iterate back into U
    return finish_info(c, info, code, total_it, outer, rel, ms, launches + (prec == MOFEM_FP64 ? 0 : 1));
}

mofem_status solver_init(mofem_ctx* c, cudaStream_t st) { return ensure_common(c, st); }

// Operator-apply tile height (rows per CTA of one wave / div, div in 1..2).  The captured
// iteration graphs hold the old grid, so they are dropped and rebuilt on next use.
mofem_status set_apply_seg_div(mofem_ctx* c, int div) {
    if (div < 1 || div > 2) return MOFEM_ERR_INVALID_ARG;
    if (c->apply_seg_div == div) return MOFEM_OK;
    c->apply_seg_div = div;
    for (int i = 0; i < 4; ++i) {
        if (c->it_graph[i]) cudaGraphExecDestroy(c->it_graph[i]);
        if (c->loop_graph[i]) cudaGraphExecDestroy(c->loop_graph[i]);
        c->it_graph[i] = nullptr;
        c->loop_graph[i] = nullptr;
        c->it_graph_max_iter[i] = 0;
    }
    return MOFEM_OK;
}

// ---- heterogeneous batches in lockstep ------------------------------------------------
// Groups of different (k, n, bc) iterate together: one CUDA graph per inner solve whose
// conditional WHILE body holds, per iteration, every group's apply and update (one branch
// per group, running side by side) and ONE persistent tensor-core launch with the four
// preconditioner GEMMs of all groups (tc_multi_launch), then a control kernel that keeps
// the loop going while any instance of any group is active.  The refinement steps are
// taken in lockstep too; a group whose instances have all converged keeps zero residuals,
// so its kernels return at once.
void fused_free(FusedState* f) {
    if (!f) return;
    if (f->loop) cudaGraphExecDestroy(f->loop);
    tc_multi_free(&f->mc);
    for (auto s : f->br) cudaStreamDestroy(s);
    for (auto e : f->ev) cudaEventDestroy(e);
    if (f->cap) cudaStreamDestroy(f->cap);
    cudaFree(f->d_scs);
    cudaFree(f->d_bat);
    *f = FusedState{};
}

mofem_status launch_set_cond_any(PcgScalars* const* scs, const int* batch, int ngroups, cudaGraphConditionalHandle h,
                                 cudaStream_t st);

static mofem_status build_fused_graph(mofem_ctx* const* cs, int G, mofem_precision pe, int max_iter, bool fixed,
                                      FusedState* f) {
    if (f->loop && f->pe == (int)pe && f->max_iter == max_iter && f->fixed == fixed) return MOFEM_OK;
    if (f->loop) {
        cudaGraphExecDestroy(f->loop);
        f->loop = nullptr;
    }
    if (!f->cap) MOFEM_CUDA_TRY(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking));
    while ((int)f->br.size() < G) {
        cudaStream_t s2;
        MOFEM_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        f->br.push_back(s2);
    }
    while ((int)f->ev.size() < G + 2) {
        cudaEvent_t e;
        MOFEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        f->ev.push_back(e);
    }
    cudaGraph_t g;
    MOFEM_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    MOFEM_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    MOFEM_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MOFEM_CUDA_TRY(cudaStreamBeginCaptureToGraph(f->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    mofem_status st = MOFEM_OK;
    for (int it = 0; it < 2 && st == MOFEM_OK; ++it) {
        // fork: every group's apply and update on its own branch
        if (cudaEventRecord(f->ev[G], f->cap) != cudaSuccess) st = MOFEM_ERR_CUDA;
        for (int gi = 0; gi < G && st == MOFEM_OK; ++gi) {
            if (cudaStreamWaitEvent(f->br[gi], f->ev[G], 0) != cudaSuccess) st = MOFEM_ERR_CUDA;
            if (st == MOFEM_OK) st = pcg_iteration(cs[gi], pe, it, max_iter, fixed, nullptr, f->br[gi], false);
            if (st == MOFEM_OK && cudaEventRecord(f->ev[gi], f->br[gi]) != cudaSuccess) st = MOFEM_ERR_CUDA;
            if (st == MOFEM_OK && cudaStreamWaitEvent(f->cap, f->ev[gi], 0) != cudaSuccess) st = MOFEM_ERR_CUDA;
        }
        // join, then the preconditioner of every group in one launch
        if (st == MOFEM_OK) st = tc_multi_launch(f->mc, f->cap);
    }
    if (st == MOFEM_OK) st = launch_set_cond_any(f->d_scs, f->d_bat, G, h, f->cap);
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(f->cap, &out);
    if (st != MOFEM_OK || ce != cudaSuccess) {
        cudaGraphDestroy(g);
        if (st == MOFEM_OK) mofem_set_last_error(cudaGetErrorString(ce), __FILE__, __LINE__);
        return st != MOFEM_OK ? st : MOFEM_ERR_CUDA;
    }
    f->body_kernels = count_kernel_nodes(body);
    cudaGraphExec_t ex;
    MOFEM_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    f->loop = ex;
    f->pe = (int)pe;
    f->max_iter = max_iter;
    f->fixed = fixed;
    return MOFEM_OK;
}

mofem_status solve_fused(mofem_ctx* const* cs, int G, const double* const* F, double* const* U, double rtol,
                         int max_iter, mofem_precision prec, FusedState* f, mofem_solve_info* infos, cudaStream_t st) {
    if (G < 1 || prec == MOFEM_FP64) return MOFEM_ERR_UNSUPPORTED;
    const mofem_precision pe = prec;
    const int which = plan_of(pe);
    for (int gi = 0; gi < G; ++gi)
        if (cs[gi]->div_product && pe == MOFEM_MIXED_FP16) return MOFEM_ERR_UNSUPPORTED;
    const bool fixed = (cs[0]->opts.flags & MOFEM_FLAG_FIXED_ITERS) != 0;
    const bool trace = getenv("MOFEM_TRACE") != nullptr;
    // ---- per-group set-up (first call allocates) and the multi-group descriptors
    for (int gi = 0; gi < G; ++gi) {
        mofem_ctx* c = cs[gi];
        MOFEM_TRY(ensure_common(c, st));
        MOFEM_TRY(ensure_w32(c, st));
        MOFEM_TRY(tc_prepare(c, which, st));
        MOFEM_TRY(ensure_apply_maps(c, false));
    }
    if (f->mc.ngroups != G || f->mc.which != which) {
        tc_multi_free(&f->mc);
        std::vector<TcGroupArgs> ga(G);
        for (int gi = 0; gi < G; ++gi)
            ga[gi] = TcGroupArgs{cs[gi], w32(cs[gi], W32_R), w32(cs[gi], W32_Z), extras()[cs[gi]].rz_slots[0]};
        MOFEM_TRY(tc_multi_build(ga.data(), G, which, &f->mc));
        cudaFree(f->d_scs);
        cudaFree(f->d_bat);
        f->d_scs = nullptr;
        f->d_bat = nullptr;
        std::vector<PcgScalars*> scs(G);
        std::vector<int> bat(G);
        for (int gi = 0; gi < G; ++gi) {
            scs[gi] = cs[gi]->d_sc;
            bat[gi] = cs[gi]->batch;
        }
        MOFEM_CUDA_TRY(cudaMalloc(&f->d_scs, sizeof(PcgScalars*) * G));
        MOFEM_CUDA_TRY(cudaMalloc(&f->d_bat, sizeof(int) * G));
        MOFEM_CUDA_TRY(cudaMemcpy(f->d_scs, scs.data(), sizeof(PcgScalars*) * G, cudaMemcpyHostToDevice));
        MOFEM_CUDA_TRY(cudaMemcpy(f->d_bat, bat.data(), sizeof(int) * G, cudaMemcpyHostToDevice));
        if (f->loop) {
            cudaGraphExecDestroy(f->loop);
            f->loop = nullptr;
        }
    }
    MOFEM_TRY(build_fused_graph(cs, G, pe, max_iter, fixed, f));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MOFEM_CUDA_TRY(cudaEventCreate(&e0));
    MOFEM_CUDA_TRY(cudaEventCreate(&e1));
    MOFEM_CUDA_TRY(cudaEventRecord(e0, st));
    // ---- right-hand sides, norms, first residuals (as solve_core, per group)
    struct GS {
        std::vector<double> bb, rr, ref2;
        double rel = 0.0;
        bool zero_guess = true, df_update = true, stalled = false, done = false;
        int total_it = 0, outer = 0;
        long long launches = 0;
        int status = 0;
    };
    std::vector<GS> gs(G);
    auto rel_max = [&](const GS& g, const std::vector<double>& r) {
        double m = 0.0;
        for (size_t i = 0; i < r.size(); ++i) {
            double v;
            if (!std::isfinite(g.ref2[i]) || !std::isfinite(r[i])) v = NAN;
            else v = g.ref2[i] > 0 ? std::sqrt(r[i] / g.ref2[i]) : (r[i] > 0 ? INFINITY : 0.0);
            if (!(v <= m)) m = v;
        }
        return m;
    };
    for (int gi = 0; gi < G; ++gi) {
        mofem_ctx* c = cs[gi];
        Extra& e = extras()[c];
        GS& g = gs[gi];
        const int B = c->batch, q = c->q;
        const long long bs = (long long)per(c);
        MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
        MOFEM_TRY(op_rhs(c, F[gi], c->Bm64, bs, c->ld, st));
        std::vector<double> both, uu;
        MOFEM_TRY(launch_dot_partials(c->Bm64, c->Bm64, true, bs, bs, B, e.bb_part, c->part.n_rz, st));
        MOFEM_TRY(launch_dot_partials(U[gi], U[gi], true, (long long)q * q, (long long)q * q, B,
                                      e.bb_part + (size_t)B * c->part.n_rz, c->part.n_rz, st));
        MOFEM_TRY(sum_partials(e.bb_part, c->part.n_rz, 2 * B, both, st));
        g.bb.assign(both.begin(), both.begin() + B);
        uu.assign(both.begin() + B, both.end());
        for (int i = 0; i < B; ++i) g.zero_guess = g.zero_guess && uu[i] == 0.0;
        if (g.zero_guess) {
            MOFEM_CUDA_TRY(cudaMemcpyAsync(c->R64, c->Bm64, sizeof(double) * bs * B, cudaMemcpyDeviceToDevice, st));
            g.rr = g.bb;
        } else {
            MOFEM_TRY(op_residual64(c, U[gi], (long long)q * q, q, c->R64, e.res_part, st));
            MOFEM_TRY(sum_partials(e.res_part, e.n_res, B, g.rr, st));
        }
        g.ref2 = g.bb;
        g.rel = rel_max(g, g.rr);
        g.launches = 1 + 2 + (g.zero_guess ? 0 : 1) + 1;
        const double floor_est = std::max(1e-11, 2.0 * 0x1p-53 * (double)q * q / (M_PI * M_PI));
        g.df_update = (c->opts.flags & MOFEM_FLAG_TRUE_RESIDUAL) == 0;
        for (int i = 0; i < B; ++i) g.df_update = g.df_update && rtol * rtol * g.ref2[i] >= floor_est * floor_est * g.bb[i];
        MOFEM_TRY(launch_convert(U[gi], 1, (long long)q * q, q, c->U64m, 1, bs, c->ld, q, q, B, st));
        g.done = g.rel <= rtol || !std::isfinite(g.rel);
    }
    const int max_outer = cs[0]->opts.max_outer > 0 ? cs[0]->opts.max_outer : 20;
    const double eta0 = cs[0]->opts.inner_rtol > 0 ? cs[0]->opts.inner_rtol : 1e-5;
    std::vector<PcgScalars> sc;
    int outer = 0;
    long long shared_launches = 0;
    auto any_open = [&]() {
        for (auto& g : gs)
            if (!g.done) return true;
        return false;
    };
    while (any_open() && outer < max_outer) {
        // ---- inner start of every group (converged groups get zero residuals: inactive)
        for (int gi = 0; gi < G; ++gi) {
            mofem_ctx* c = cs[gi];
            GS& g = gs[gi];
            const int B = c->batch, q = c->q;
            const long long bs = (long long)per(c);
            double eta = std::max(g.outer == 0 ? eta0 : 0.1 * eta0, 0.3 * rtol / std::max(g.rel, 1e-300));
            if (eta >= 1.0) eta = 0.5;
            MOFEM_TRY(launch_convert(c->R64, 1, bs, c->ld, w32(c, W32_R), 0, bs, c->ld, q, q, B, st));
            for (int i = 0; i < B; ++i) {
                const double ri = g.ref2[i] > 0 ? std::sqrt(g.rr[i] / g.ref2[i]) : 0.0;
                if (g.done || ri <= rtol)
                    MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_R) + bs * i, 0, sizeof(float) * bs, st));
            }
            MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_U), 0, sizeof(float) * bs * B, st));
            MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_ULO), 0, sizeof(float) * bs * B, st));
            MOFEM_CUDA_TRY(cudaMemsetAsync(w32(c, W32_QB), 0, sizeof(float) * bs * B, st));
            MOFEM_TRY(launch_dot_partials(w32(c, W32_R), w32(c, W32_R), false, bs, bs, B, c->part.rr, c->part.n_upd, st));
            MOFEM_TRY(launch_pcg_init(c, c->part.rr, c->part.n_upd, nullptr, eta, st));
            if (which == 2)
                MOFEM_TRY(launch_convert_scaled_f16(w32(c, W32_R), bs, c->ld, c->tc[2].Rop, bs, c->ld, q, q, B, c->d_sc,
                                                    st));
            else
                MOFEM_TRY(launch_convert(w32(c, W32_R), 0, bs, c->ld, c->tc[which].Rop, conv_kind_of_plan(which), bs,
                                         c->ld, q, q, B, st));
        }
        MOFEM_TRY(tc_multi_launch(f->mc, st));   // Z0 and <R0, Z0> of every group
        MOFEM_CUDA_TRY(cudaGraphLaunch(f->loop, st));
        // ---- fold, residual update and norms of every open group
        int max_it = 0;
        for (int gi = 0; gi < G; ++gi) {
            mofem_ctx* c = cs[gi];
            Extra& e = extras()[c];
            GS& g = gs[gi];
            const int B = c->batch, q = c->q;
            const long long bs = (long long)per(c);
            MOFEM_TRY(read_scalars(c, sc, st));
            int it = 0;
            bool bad = false;
            for (auto& x : sc) {
                it = std::max(it, x.iters);
                bad = bad || (x.status & DEV_ERR_NONFINITE) || !std::isfinite(x.rr);
            }
            max_it = std::max(max_it, it);
            if (g.done) continue;
            if (bad && pe == MOFEM_MIXED_FP16) {   // FP16 range exceeded: the caller solves the groups one by one
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return MOFEM_ERR_UNSUPPORTED;
            }
            const bool from_zero = g.outer == 0 && g.zero_guess;
            const bool upd = g.df_update && (!from_zero || residual_update_dfd_ok(c));
            const int dmode = !upd ? 0 : (from_zero ? 2 : 1);
            MOFEM_TRY(launch_fold_df(c->U64m, w32(c, W32_U), w32(c, W32_ULO), bs, B, c->d_sc, w32(c, W32_QA), dmode, st));
            g.total_it += it;
            g.launches += 8 + 3;   // convert, zeroing, dot, init, operand copy; fold, residual
            int nblk = 0;
            mofem_status du = MOFEM_ERR_UNSUPPORTED;
            if (upd)
                du = from_zero ? launch_residual_update_dfd(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, e.res_part, &nblk, st)
                               : launch_residual_update_df(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, e.res_part, &nblk, st);
            if (du == MOFEM_OK) {
                MOFEM_TRY(sum_partials(e.res_part, nblk, B, g.rr, st));
            } else {
                if (du != MOFEM_ERR_UNSUPPORTED) return du;
                MOFEM_TRY(op_residual64(c, c->U64m, bs, c->ld, c->R64, e.res_part, st));
                MOFEM_TRY(sum_partials(e.res_part, e.n_res, B, g.rr, st));
            }
            const double prev = g.rel;
            g.rel = rel_max(g, g.rr);
            ++g.outer;
            if (std::isfinite(g.rel) && g.rel > 0.5 * prev) g.stalled = true;
            g.done = g.rel <= rtol || !std::isfinite(g.rel) || g.stalled || fixed;
            (void)q;
        }
        // one tensor-core launch and one graph per inner solve, plus the bodies of two iterations
        shared_launches += 1 + (long long)std::max(1, (max_it + 1) / 2) * f->body_kernels;
        if (trace) fprintf(stderr, "[mofem] fused outer %d: inner iterations %d\n", outer + 1, max_it);
        ++outer;
    }
    MOFEM_CUDA_TRY(cudaEventRecord(e1, st));
    std::vector<int> dev_status(G, 0);
    for (int gi = 0; gi < G; ++gi) {
        mofem_ctx* c = cs[gi];
        const int q = c->q;
        MOFEM_TRY(launch_convert(c->U64m, 1, (long long)per(c), c->ld, U[gi], 1, (long long)q * q, q, q, q, c->batch, st));
        MOFEM_CUDA_TRY(cudaMemcpyAsync(&dev_status[gi], c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mofem_status worst = MOFEM_OK;
    for (int gi = 0; gi < G; ++gi) {
        GS& g = gs[gi];
        mofem_status code = MOFEM_OK;
        if (dev_status[gi] & DEV_ERR_TIMEOUT) code = MOFEM_ERR_TIMEOUT;
        else if (!std::isfinite(g.rel)) code = MOFEM_ERR_NONFINITE;
        else if (!(g.rel <= rtol) && !fixed) code = MOFEM_ERR_NOT_CONVERGED;
        if (infos) {
            mofem_solve_info& in = infos[gi];
            in.status = code;
            in.iterations = g.total_it;
            in.outer_steps = g.outer;
            in.batch = cs[gi]->batch;
            in.rel_residual = g.rel;
            in.ms_total = ms;
            in.kernel_launches = g.launches + shared_launches;   // the shared launches counted in every group
        }
        if (code != MOFEM_OK && (worst == MOFEM_OK || worst == MOFEM_ERR_NOT_CONVERGED)) worst = code;
    }
    return worst;
}

mofem_status solve_elliptic(mofem_ctx* c, const double* F, double* U, double rtol, int max_iter, mofem_precision prec,
                            mofem_solve_info* info, cudaStream_t st) {
    MOFEM_TRY(ensure_common(c, st));
    MOFEM_TRY(op_rhs(c, F, c->Bm64, (long long)per(c), c->ld, st));
    const mofem_status r = solve_core(c, U, (long long)c->q * c->q, c->q, rtol, max_iter, prec, 0, info, st);
    if (info) info->kernel_launches += 1;   // the right-hand side
    return r;
}

mofem_status solve_imex(mofem_ctx* c, double d_u, double tau, const double* Un, const double* Fn, double* Unp1,
                        double rtol, mofem_precision prec, mofem_solve_info* info, cudaStream_t st, double cu) {
    MOFEM_TRY(ensure_common(c, st));
    double* Fbar = nullptr;
    const long long nn = (long long)c->n * c->n, qq0 = (long long)c->q * c->q;
    MOFEM_CUDA_TRY(cudaMallocAsync((void**)&Fbar, sizeof(double) * (size_t)nn * c->batch, st));
    // nodal gamma_i (cu U_n + tau F_n) per instance (each instance its own diffusion d_i = 1/(gamma_i tau))
    mofem_status s = MOFEM_OK;
    for (int i = 0; i < c->batch && s == MOFEM_OK; ++i)
        s = launch_imex_rhs(Un + qq0 * i, Fn + nn * i, Fbar + nn * i, c->n, c->q, c->off, c->gamma[i], tau, cu, 1,
                            st);
    if (s == MOFEM_OK) s = op_rhs(c, Fbar, c->Bm64, (long long)per(c), c->ld, st);
    cudaFreeAsync(Fbar, st);
    MOFEM_TRY(s);
    (void)d_u;
    const long long qq = (long long)c->q * c->q;
    if (Unp1 != Un)
        MOFEM_CUDA_TRY(cudaMemcpyAsync(Unp1, Un, sizeof(double) * qq * c->batch, cudaMemcpyDeviceToDevice, st));
    // rtol > 0: ||B - S U||_F <= rtol ||B||_F; else the paper's ||R_s|| <= tau ||R_0|| (Sec. 6)
    const mofem_status r = rtol > 0 ? solve_core(c, Unp1, qq, c->q, rtol, 100000, prec, 0, info, st)
                                    : solve_core(c, Unp1, qq, c->q, tau, 100000, prec, 1, info, st);
    if (info) info->kernel_launches += c->batch + 1;   // the nodal load per instance and the right-hand side
    return r;
}

// One backward step of the discrete adjoint of solve_imex with a nodal source F and an
// explicit linear reaction -r u:  S U_np1 = (1 - tau r) M~ U_n + tau M~_all F,
// S = M~ + d_u tau A~ = d_u tau L with L the handle's operator (gamma = 1/(d_u tau)):
//   Y = S^{-1} Lam_np1,  Lam_n = (1 - tau r) M~ Y,  dF += tau M~_all^T Y,
//   dr[i] = -tau <Y, M~ U_n>,  dd[i] = -tau <Y, A~ U_np1> = -tau (<Y, L U_np1> - gamma <Y, M~ U_np1>).
// M~_all^T Y = M_s pad(Y) M_t^T with the untrimmed masses (pad: zero boundary rows and columns).
mofem_status solve_imex_adjoint(mofem_ctx* c, double d_u, double tau, double r, const double* Lam1, const double* U0,
                                const double* U1, double* Lam0, double* Y_io, double* dF, double* dd, double* dr,
                                double rtol, mofem_precision prec, mofem_solve_info* info, cudaStream_t st) {
    MOFEM_TRY(ensure_common(c, st));
    Extra& e = extras()[c];
    const int q = c->q, B = c->batch, n = c->n;
    const long long qq = (long long)q * q, nn = (long long)n * n;
    double* buf = nullptr;
    const size_t nbuf = (size_t)qq * B * 3 + (dF ? (size_t)nn * B * 2 : 0);
    MOFEM_CUDA_TRY(cudaMallocAsync((void**)&buf, sizeof(double) * nbuf, st));
    double *Y = Y_io ? Y_io : buf, *LU = buf + qq * B, *MU = buf + 2 * qq * B;
    double *Ypad = buf + 3 * qq * B, *G = Ypad + nn * B;
    mofem_status s = launch_scale_copy64(Lam1, qq, q, c->Bm64, (long long)per(c), c->ld, q, q, B, 1.0 / (d_u * tau), st);
    if (s == MOFEM_OK && !Y_io)   // no guess: start from zero
        s = cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)qq * B, st) == cudaSuccess ? MOFEM_OK : MOFEM_ERR_CUDA;
    mofem_status solve = MOFEM_OK;
    if (s == MOFEM_OK) {
        solve = solve_core(c, Y, qq, q, rtol, 100000, prec, 0, info, st);
        if (solve != MOFEM_OK && solve != MOFEM_ERR_NOT_CONVERGED) s = solve;
    }
    long long launches = 6;
    if (s == MOFEM_OK) s = op_mass(c, Y, qq, q, Lam0, qq, q, st);
    if (s == MOFEM_OK && r != 0.0) {
        s = launch_scale_copy64(Lam0, qq, q, Lam0, qq, q, q, q, B, 1.0 - tau * r, st);
        launches += 1;
    }
    if (s == MOFEM_OK) s = op_apply(c, true, U1, qq, q, LU, qq, q, nullptr, st);
    if (s == MOFEM_OK) s = op_mass(c, U1, qq, q, MU, qq, q, st);
    std::vector<double> both;   // <Y, L U_np1>, <Y, M~ U_np1> [, <Y, M~ U_n>], read back with one synchronisation
    const int nd = dr ? 3 : 2;
    if (s == MOFEM_OK) s = launch_dot_partials(Y, LU, true, qq, qq, B, e.bb_part, c->part.n_rz, st);
    if (s == MOFEM_OK) s = launch_dot_partials(Y, MU, true, qq, qq, B, e.bb_part + (size_t)B * c->part.n_rz, c->part.n_rz, st);
    if (s == MOFEM_OK && dr) {
        // the third product needs its own partial slice: reuse LU's storage once <Y, L U> is summed
        s = sum_partials(e.bb_part, c->part.n_rz, 2 * B, both, st);
        if (s == MOFEM_OK) s = op_mass(c, U0, qq, q, MU, qq, q, st);
        if (s == MOFEM_OK) s = launch_dot_partials(Y, MU, true, qq, qq, B, e.bb_part, c->part.n_rz, st);
        std::vector<double> third;
        if (s == MOFEM_OK) s = sum_partials(e.bb_part, c->part.n_rz, B, third, st);
        if (s == MOFEM_OK) both.insert(both.end(), third.begin(), third.end());
        launches += 2;
    } else if (s == MOFEM_OK) {
        s = sum_partials(e.bb_part, c->part.n_rz, 2 * B, both, st);
    }
    if (s == MOFEM_OK && dF) {
        // dF += tau M_s pad(Y) M_t^T (untrimmed masses; the generic apply with one mass term)
        s = cudaMemsetAsync(Ypad, 0, sizeof(double) * (size_t)nn * B, st) == cudaSuccess ? MOFEM_OK : MOFEM_ERR_CUDA;
        if (s == MOFEM_OK)
            s = launch_convert(Y, 1, qq, q, Ypad + (size_t)c->off * n + c->off, 1, nn, n, q, q, B, st);
        if (s == MOFEM_OK) {
            ApplyArgs a{};
            a.X = Ypad; a.x_bs = nn; a.x_ld = n;
            a.Y = G; a.y_bs = nn; a.y_ld = n;
            a.S = c->Smf64; a.s_bs = (long long)c->P * n; a.T = c->Tmf64;
            a.rows_in = a.cols_in = a.rows_out = a.cols_out = n;
            a.off = 0;
            s = launch_apply(c->K, 1, true, APPLY_PLAIN, a, B, st);
        }
        if (s == MOFEM_OK) s = launch_axpy64(G, nn, n, dF, nn, n, n, n, B, tau, st);
        launches += 3;
    }
    cudaFreeAsync(buf, st);
    MOFEM_TRY(s);
    for (int i = 0; i < B; ++i) {
        dd[i] = -tau * (both[i] - c->gamma[i] * both[B + i]);
        if (dr) dr[i] = -tau * both[2 * B + i];
    }
    if (info) info->kernel_launches += launches;
    return solve;
}

// Benchmark hook: repeated launches of one hot kernel on internal buffers.
// One search-direction step on caller buffers (the solver's first kernel of an
// iteration): Q = Z + beta Q_prev, LQ = L(Q), alpha = rz / <Q, LQ>.
mofem_status pcg_direction(mofem_ctx* c, const void* Z, const void* Qp, const double* beta, const double* rz,
                           void* Q, void* LQ, int ld, double* alpha, bool fp64, cudaStream_t st) {
    MOFEM_TRY(ensure_common(c, st));
    Extra& e = extras()[c];
    const int B = c->batch, esz = fp64 ? 8 : 4;
    if (!e.dir_sc) MOFEM_CUDA_TRY(cudaMalloc(&e.dir_sc, sizeof(PcgScalars) * B));
    const int WCT = 128 + 8;
    const int HR = apply_pcg_box_rows(c->K, c->NT, fp64);
    CUtensorMap mZ, mQ, mS;
    MOFEM_TRY(make_row_map(&mZ, Z, esz, c->q, c->q, B, ld, WCT, HR));
    MOFEM_TRY(make_row_map(&mQ, Qp, esz, c->q, c->q, B, ld, WCT, HR));
    const bool packed = apply_pcg_packed(c->K, c->NT, fp64);
    if (packed)
        MOFEM_TRY(make_row_map(&mS, c->Srow32, 4, c->s_row, c->q, B, c->s_row, c->s_row, apply_pcg_s_box_rows()));
    std::vector<PcgScalars> h(B);
    for (int i = 0; i < B; ++i) {
        h[i] = PcgScalars{};
        h[i].rz = rz[i];
        h[i].beta = beta[i];
        h[i].iters = 1;   // > 0: the kernel applies beta
        h[i].active = 1;
    }
    MOFEM_CUDA_TRY(cudaMemcpyAsync(e.dir_sc, h.data(), sizeof(PcgScalars) * B, cudaMemcpyHostToDevice, st));
    MOFEM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), st));
    ApplyPcgArgs a{};
    a.S = fp64 ? (const void*)c->S64 : (const void*)c->S32;
    a.s_bs = (long long)c->NT * c->P * c->q;
    a.T = fp64 ? (const void*)c->T64 : (const void*)c->T32;
    a.q = c->q; a.ld = ld; a.bs = (long long)ld * c->q;
    a.Qnew = Q; a.LQ = LQ;
    a.partial = c->part.qlq; a.counter = c->d_ctr + 3 * B;
    a.sc = e.dir_sc; a.use_sc = 1;
    a.status = c->d_status;
    a.seg_div = c->apply_seg_div;
    MOFEM_TRY(launch_apply_pcg(c->K, c->NT, fp64, mZ, mQ, packed ? &mS : nullptr, a, B, st));
    MOFEM_CUDA_TRY(cudaMemcpyAsync(h.data(), e.dir_sc, sizeof(PcgScalars) * B, cudaMemcpyDeviceToHost, st));
    int dev_status = 0;
    MOFEM_CUDA_TRY(cudaMemcpyAsync(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    int sc_status = 0;
    for (int i = 0; i < B; ++i) {
        alpha[i] = h[i].alpha;
        sc_status |= h[i].status;
    }
    if (dev_status & DEV_ERR_TIMEOUT) {
        mofem_set_last_error("operator apply: a TMA staging wait timed out", __FILE__, __LINE__);
        return MOFEM_ERR_TIMEOUT;
    }
    if (sc_status & DEV_ERR_NONFINITE) return MOFEM_ERR_NONFINITE;
    if (sc_status & DEV_ERR_BREAKDOWN) return MOFEM_ERR_BREAKDOWN;
    return MOFEM_OK;
}

mofem_status bench_kernel(mofem_ctx* c, int kernel, mofem_precision prec, int reps, cudaStream_t st) {
    MOFEM_TRY(ensure_common(c, st));
    const long long bs = (long long)per(c);
    const int which = plan_of(prec);
    if (kernel == 6) {
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(op_residual64(c, c->Bm64, bs, c->ld, c->R64, extras()[c].res_part, st));
        return MOFEM_OK;
    }
    MOFEM_TRY(ensure_w32(c, st));
    if (kernel >= 1 && kernel <= 4) {
        MOFEM_TRY(tc_prepare(c, which, st));
        for (int r = 0; r < reps; ++r) MOFEM_TRY(tc_gemm_one(c, which, kernel - 1, w32(c, W32_Z), st));
        return MOFEM_OK;
    }
    if (kernel == 0) {
        MOFEM_TRY(ensure_apply_maps(c, false));
        Extra& e = extras()[c];
        ApplyPcgArgs a{};
        a.S = c->S32; a.s_bs = (long long)c->NT * c->P * c->q; a.T = c->T32;
        a.q = c->q; a.ld = c->ld; a.bs = bs;
        a.Qnew = w32(c, W32_QA); a.LQ = w32(c, W32_LQ);
        a.partial = c->part.qlq; a.counter = c->d_ctr + 3 * c->batch;
        a.sc = c->d_sc; a.use_sc = 0;
        a.status = c->d_status;
        a.seg_div = c->apply_seg_div;
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(launch_apply_pcg(c->K, c->NT, false, e.mZ32, e.mQB32, &e.mS32, a, c->batch, st));
        return MOFEM_OK;
    }
    if (kernel == 5 || kernel == 7) {   // residual update of an even (5) or odd (7) iteration, FP16 operand copy
        MOFEM_TRY(tc_prepare(c, 2, st));
        const bool packed = apply_pcg_packed(c->K, c->NT, false);
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(launch_pcg_update(c, false, w32(c, W32_U), w32(c, W32_ULO), w32(c, W32_R), w32(c, W32_QA),
                                        w32(c, W32_LQ), w32(c, W32_Z), c->tc[2].Rop, 2, packed ? 0 : 1, 1 << 30, true,
                                        nullptr, st, false, w32(c, W32_QB), kernel == 7 ? 1 : 0));
        return MOFEM_OK;
    }
    if (kernel == 9) {   // the preconditioner's four GEMMs as one chained launch (<R, Z> partials, no beta)
        MOFEM_TRY(tc_prepare(c, which, st));
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(tc_precond(c, which, w32(c, W32_R), bs, c->ld, w32(c, W32_Z), c->ld, bs, extras()[c].rz_slots[0],
                                 nullptr, st, true));
        return MOFEM_OK;
    }
    if (kernel == 10) {   // the same update in difference form (the step from zero)
        int nblk = 0;
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(launch_residual_update_dfd(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, extras()[c].res_part,
                                                 &nblk, st));
        return MOFEM_OK;
    }
    if (kernel == 11) {   // the FP64 form's preconditioner: four cuBLAS DGEMMs per instance + division
        MOFEM_TRY(ensure_w64(c, st));
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(precond64(c, w64(c, W64_R), bs, c->ld, w64(c, W64_Z), bs, c->ld, st));
        return MOFEM_OK;
    }
    if (kernel == 8) {   // double-float residual update of a refinement step
        int nblk = 0;
        for (int r = 0; r < reps; ++r)
            MOFEM_TRY(launch_residual_update_df(c, w32(c, W32_U), w32(c, W32_ULO), c->R64, extras()[c].res_part,
                                                &nblk, st));
        return MOFEM_OK;
    }
    return MOFEM_ERR_INVALID_ARG;
}
