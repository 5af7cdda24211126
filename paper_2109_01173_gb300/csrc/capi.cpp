// extern "C" entry points of libmofem (declared in include/mofem.h): argument
// validation, handle lifetime, dispatch to the setup, kernels and solver.
#include "internal.h"

#include <cmath>
#include <new>

namespace {

mofem_opts default_opts(const mofem_opts* o) {
    mofem_opts d{};
    if (o) d = *o;
    if (d.max_outer <= 0) d.max_outer = 20;
    if (!(d.inner_rtol > 0.0)) d.inner_rtol = 1e-5;
    return d;
}

bool valid_precision(mofem_precision p) {
    return p == MOFEM_FP64 || p == MOFEM_MIXED_TF32 || p == MOFEM_MIXED_BF16 || p == MOFEM_MIXED_FP16;
}

}  // namespace

extern "C" {

const char* mofem_status_string(mofem_status s) {
    switch (s) {
        case MOFEM_OK: return "MOFEM_OK";
        case MOFEM_ERR_INVALID_ARG: return "MOFEM_ERR_INVALID_ARG";
        case MOFEM_ERR_CUDA: return "MOFEM_ERR_CUDA";
        case MOFEM_ERR_EIG: return "MOFEM_ERR_EIG";
        case MOFEM_ERR_NONFINITE: return "MOFEM_ERR_NONFINITE";
        case MOFEM_ERR_BREAKDOWN: return "MOFEM_ERR_BREAKDOWN";
        case MOFEM_ERR_NOT_CONVERGED: return "MOFEM_ERR_NOT_CONVERGED";
        case MOFEM_ERR_TIMEOUT: return "MOFEM_ERR_TIMEOUT";
        case MOFEM_ERR_OOM: return "MOFEM_ERR_OOM";
        case MOFEM_ERR_UNSUPPORTED: return "MOFEM_ERR_UNSUPPORTED";
    }
    return "MOFEM_ERR_?";
}

mofem_status mofem_setup_batched(int batch, const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                                 const double* gamma, mofem_bc bc, const mofem_opts* opts, cudaStream_t stream,
                                 mofem_handle* out) {
    if (!out || !g1 || !g2 || !gamma || batch < 1) return MOFEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 0 || k > 4) return MOFEM_ERR_INVALID_ARG;
    if (bc != MOFEM_BC_DIRICHLET && bc != MOFEM_BC_NEUMANN) return MOFEM_ERR_INVALID_ARG;
    const int d = k == 0 ? 1 : k;
    if (n_nodes < 3 || (n_nodes - 1) % d != 0 || n_nodes > 16385) return MOFEM_ERR_INVALID_ARG;
    for (int i = 0; i < batch; ++i) {
        if (!g1[i].g || !g1[i].dg || !g2[i].g || !g2[i].dg) return MOFEM_ERR_INVALID_ARG;
        if (!std::isfinite(gamma[i]) || gamma[i] < 0.0) return MOFEM_ERR_INVALID_ARG;
        if (bc == MOFEM_BC_NEUMANN && !(gamma[i] > 0.0)) return MOFEM_ERR_INVALID_ARG;   // singular operator
    }
    if (opts && (opts->quad_points < 0 || opts->quad_points > 16)) return MOFEM_ERR_INVALID_ARG;
    if (opts && (opts->pencil < MOFEM_PENCIL_AVERAGED || opts->pencil > MOFEM_PENCIL_AUA))
        return MOFEM_ERR_INVALID_ARG;
    if (opts && (opts->pencil == MOFEM_PENCIL_PRODUCT || opts->pencil == MOFEM_PENCIL_AUA) &&
        bc != MOFEM_BC_DIRICHLET) {
        mofem_set_last_error("single-term stiffness preconditioner: K_s[h] and K_t (+ K_t[t^2]) are singular under "
                             "Neumann BC", __FILE__, __LINE__);
        return MOFEM_ERR_INVALID_ARG;
    }
    if (opts && opts->pencil == MOFEM_PENCIL_PARABOLIC) {
        // the t-factor M_t + (K_t + K_t[t^2]) / gamma and its eigenvectors are shared by the batch
        for (int i = 0; i < batch; ++i)
            if (!(gamma[i] > 0.0) || gamma[i] != gamma[0]) {
                mofem_set_last_error("parabolic preconditioner: gamma = 1/(d_u tau) must be positive and equal in "
                                     "every instance", __FILE__, __LINE__);
                return MOFEM_ERR_INVALID_ARG;
            }
    }
    mofem_ctx* c = new (std::nothrow) mofem_ctx();
    if (!c) return MOFEM_ERR_OOM;
    c->batch = batch;
    c->k = k;
    c->n = n_nodes;
    c->bc = bc;
    c->opts = default_opts(opts);
    c->gamma.assign(gamma, gamma + batch);
    cudaGetDevice(&c->dev);
    mofem_status s = mofem_build(c, g1, g2, gamma, stream);
    if (s == MOFEM_OK) s = solver_init(c, stream);
    if (s == MOFEM_OK && cudaStreamSynchronize(stream) != cudaSuccess) s = MOFEM_ERR_CUDA;
    if (s != MOFEM_OK) {
        mofem_free_extra(c);
        mofem_free(c);
        delete c;
        return s;
    }
    *out = c;
    return MOFEM_OK;
}

mofem_status mofem_setup(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes, double gamma,
                         mofem_bc bc, const mofem_opts* opts, cudaStream_t stream, mofem_handle* out) {
    return mofem_setup_batched(1, g1, g2, k, n_nodes, &gamma, bc, opts, stream, out);
}

mofem_status mofem_get_dims(mofem_handle h, int* batch, int* n_nodes, int* q, int* n_terms) {
    if (!h) return MOFEM_ERR_INVALID_ARG;
    if (batch) *batch = h->batch;
    if (n_nodes) *n_nodes = h->n;
    if (q) *q = h->q;
    if (n_terms) *n_terms = h->NT;
    return MOFEM_OK;
}

mofem_status mofem_apply(mofem_handle h, const void* X, void* Y, int ld, mofem_precision prec, cudaStream_t stream) {
    if (!h || !X || !Y || ld < h->q || !valid_precision(prec)) return MOFEM_ERR_INVALID_ARG;
    const long long bs = (long long)ld * h->q;
    return op_apply(h, prec == MOFEM_FP64, X, bs, ld, Y, bs, ld, nullptr, stream);
}

mofem_status mofem_rhs(mofem_handle h, const double* F, double* B, int ld_b, cudaStream_t stream) {
    if (!h || !F || !B || ld_b < h->q) return MOFEM_ERR_INVALID_ARG;
    return op_rhs(h, F, B, (long long)ld_b * h->q, ld_b, stream);
}

mofem_status mofem_precond(mofem_handle h, const void* R, void* Z, int ld, mofem_precision prec, cudaStream_t stream) {
    if (!h || !R || !Z || ld < h->q || !valid_precision(prec)) return MOFEM_ERR_INVALID_ARG;
    const long long bs = (long long)ld * h->q;
    if (prec == MOFEM_FP64) return precond64(h, (const double*)R, bs, ld, (double*)Z, bs, ld, stream);
    const mofem_precision pe = (prec == MOFEM_MIXED_FP16 && h->div_product) ? MOFEM_MIXED_TF32 : prec;
    return precond_tc(h, plan_of(pe), (const float*)R, bs, ld, (float*)Z, bs, ld, nullptr, nullptr, stream);
}

mofem_status mofem_pcg_direction(mofem_handle h, const void* Z, const void* Q_prev, const double* beta,
                                 const double* rz, void* Q, void* LQ, int ld, double* alpha, mofem_precision prec,
                                 cudaStream_t stream) {
    if (!h || !Z || !Q_prev || !beta || !rz || !Q || !LQ || !alpha || ld < h->q || !valid_precision(prec))
        return MOFEM_ERR_INVALID_ARG;
    const int esz = prec == MOFEM_FP64 ? 8 : 4;
    auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
    if (((long long)ld * esz) % 16 != 0 || misaligned(Z) || misaligned(Q_prev) || misaligned(Q) || misaligned(LQ)) {
        mofem_set_last_error("mofem_pcg_direction: buffers must be 16-byte aligned with ld*size a multiple of 16",
                             __FILE__, __LINE__);
        return MOFEM_ERR_INVALID_ARG;
    }
    return pcg_direction(h, Z, Q_prev, beta, rz, Q, LQ, ld, alpha, prec == MOFEM_FP64, stream);
}

mofem_status mofem_pcg_solve(mofem_handle h, const double* F, double* U, double rtol, int max_iter,
                             mofem_precision prec, mofem_solve_info* info, cudaStream_t stream) {
    if (!h || !F || !U || !(rtol > 0.0) || max_iter < 1 || !valid_precision(prec)) return MOFEM_ERR_INVALID_ARG;
    return solve_elliptic(h, F, U, rtol, max_iter, prec, info, stream);
}

static bool imex_gamma_ok(mofem_handle h, double d_u, double tau) {
    const double want = 1.0 / (d_u * tau);
    for (int i = 0; i < h->batch; ++i)
        if (std::fabs(h->gamma[i] - want) > 1e-12 * want) return false;
    return true;
}

mofem_status mofem_imex_step(mofem_handle h, double d_u, double tau, const double* U_n, const double* F_n,
                             double* U_np1, mofem_precision prec, mofem_solve_info* info, cudaStream_t stream) {
    return mofem_imex_step_tol(h, d_u, tau, U_n, F_n, U_np1, 0.0, prec, info, stream);
}

mofem_status mofem_imex_step_tol(mofem_handle h, double d_u, double tau, const double* U_n, const double* F_n,
                                 double* U_np1, double rtol, mofem_precision prec, mofem_solve_info* info,
                                 cudaStream_t stream) {
    if (!h || !U_n || !F_n || !U_np1 || !(d_u > 0.0) || !(tau > 0.0) || !(rtol >= 0.0) || !valid_precision(prec))
        return MOFEM_ERR_INVALID_ARG;
    if (!imex_gamma_ok(h, d_u, tau)) return MOFEM_ERR_INVALID_ARG;
    return solve_imex(h, d_u, tau, U_n, F_n, U_np1, rtol, prec, info, stream);
}

mofem_status mofem_imex_adjoint_step(mofem_handle h, double d_u, double tau, const double* Lam_np1,
                                     const double* U_np1, double* Lam_n, double* Y, double* dd_u, double rtol,
                                     mofem_precision prec, mofem_solve_info* info, cudaStream_t stream) {
    if (!h || !Lam_np1 || !U_np1 || !Lam_n || !dd_u || !(d_u > 0.0) || !(tau > 0.0) || !(rtol > 0.0) ||
        !valid_precision(prec) || Lam_n == Lam_np1)
        return MOFEM_ERR_INVALID_ARG;
    if (Y && (Y == Lam_np1 || Y == Lam_n || Y == U_np1)) return MOFEM_ERR_INVALID_ARG;
    if (!imex_gamma_ok(h, d_u, tau)) return MOFEM_ERR_INVALID_ARG;
    return solve_imex_adjoint(h, d_u, tau, 0.0, Lam_np1, nullptr, U_np1, Lam_n, Y, nullptr, dd_u, nullptr, rtol, prec,
                              info, stream);
}

mofem_status mofem_imex_step_src(mofem_handle h, double d_u, double tau, double r, const double* U_n, const double* F,
                                 double* U_np1, double rtol, mofem_precision prec, mofem_solve_info* info,
                                 cudaStream_t stream) {
    if (!h || !U_n || !F || !U_np1 || !(d_u > 0.0) || !(tau > 0.0) || !(rtol >= 0.0) || !std::isfinite(r) ||
        !valid_precision(prec))
        return MOFEM_ERR_INVALID_ARG;
    if (!imex_gamma_ok(h, d_u, tau)) return MOFEM_ERR_INVALID_ARG;
    return solve_imex(h, d_u, tau, U_n, F, U_np1, rtol, prec, info, stream, 1.0 - tau * r);
}

mofem_status mofem_imex_adjoint_step_src(mofem_handle h, double d_u, double tau, double r, const double* Lam_np1,
                                         const double* U_n, const double* U_np1, double* Lam_n, double* Y, double* dF,
                                         double* dd_u, double* dr, double rtol, mofem_precision prec,
                                         mofem_solve_info* info, cudaStream_t stream) {
    if (!h || !Lam_np1 || !U_np1 || !Lam_n || !dd_u || !(d_u > 0.0) || !(tau > 0.0) || !(rtol > 0.0) ||
        !std::isfinite(r) || !valid_precision(prec) || Lam_n == Lam_np1 || (dr && !U_n))
        return MOFEM_ERR_INVALID_ARG;
    if (Y && (Y == Lam_np1 || Y == Lam_n || Y == U_np1 || Y == U_n)) return MOFEM_ERR_INVALID_ARG;
    if (!imex_gamma_ok(h, d_u, tau)) return MOFEM_ERR_INVALID_ARG;
    return solve_imex_adjoint(h, d_u, tau, r, Lam_np1, U_n, U_np1, Lam_n, Y, dF, dd_u, dr, rtol, prec, info, stream);
}

mofem_status mofem_rds_step(mofem_handle h, double tau, const double* U_n, const double* F_n, double* U_np1,
                            double rtol, mofem_precision prec, mofem_solve_info* info, cudaStream_t stream) {
    if (!h || !U_n || !F_n || !U_np1 || !(tau > 0.0) || !(rtol >= 0.0) || !valid_precision(prec))
        return MOFEM_ERR_INVALID_ARG;
    for (int i = 0; i < h->batch; ++i)
        if (!(h->gamma[i] > 0.0)) return MOFEM_ERR_INVALID_ARG;
    return solve_imex(h, 0.0, tau, U_n, F_n, U_np1, rtol, prec, info, stream);
}

mofem_status mofem_dib_kinetics(const mofem_dib_params* p, double rho, const double* eta, const double* theta,
                                double* f, double* g, long long count, cudaStream_t stream) {
    if (!p || !eta || !theta || !f || !g || count < 0 || !std::isfinite(rho)) return MOFEM_ERR_INVALID_ARG;
    return launch_dib_kinetics(*p, rho, eta, theta, f, g, count, stream);
}

mofem_status mofem_dib_equilibrium(const mofem_dib_params* p, double* eta, double* theta) {
    if (!p || !eta || !theta) return MOFEM_ERR_INVALID_ARG;
    return dib_equilibrium(*p, eta, theta);
}

mofem_status mofem_dib_run(mofem_handle h, const mofem_dib_params* p, double rho, double tau, int n_steps,
                           double* U, double rtol, mofem_precision prec, double* incr, mofem_solve_info* info,
                           cudaStream_t stream) {
    if (!h || !p || !U || !(tau > 0.0) || n_steps < 0 || !(rtol >= 0.0) || !valid_precision(prec) ||
        !std::isfinite(rho))
        return MOFEM_ERR_INVALID_ARG;
    if (h->batch != 2 || h->q != h->n || !(p->d_theta > 0.0)) {
        mofem_set_last_error("mofem_dib_run: needs a Neumann handle with two instances (eta, theta)", __FILE__,
                             __LINE__);
        return MOFEM_ERR_INVALID_ARG;
    }
    const double ge = 1.0 / tau, gt = 1.0 / (p->d_theta * tau);
    if (std::fabs(h->gamma[0] - ge) > 1e-12 * ge || std::fabs(h->gamma[1] - gt) > 1e-12 * gt) {
        mofem_set_last_error("mofem_dib_run: handle gamma must be {1/tau, 1/(d_theta tau)}", __FILE__, __LINE__);
        return MOFEM_ERR_INVALID_ARG;
    }
    return dib_run(h, *p, rho, tau, n_steps, U, rtol, prec, incr, info, stream);
}

mofem_status mofem_bench_kernel(mofem_handle h, int kernel, mofem_precision prec, int reps, cudaStream_t stream) {
    if (!h || kernel < 0 || kernel > 11 || reps < 0 || !valid_precision(prec)) return MOFEM_ERR_INVALID_ARG;
    if (kernel >= 1 && kernel <= 4 && prec == MOFEM_FP64) return MOFEM_ERR_INVALID_ARG;
    return bench_kernel(h, kernel, prec, reps, stream);
}

mofem_status mofem_get_eigen(mofem_handle h, double* Q1, double* Q2, double* lambda, double* mu,
                             int* divisor_product, cudaStream_t stream) {
    if (!h) return MOFEM_ERR_INVALID_ARG;
    const int q = h->q, ld = h->ld, B = h->batch;
    const size_t w = sizeof(double) * q, lw = sizeof(double) * ld;
    if (Q1)
        MOFEM_CUDA_TRY(cudaMemcpy2DAsync(Q1, w, h->Q1_64, lw, w, (size_t)q * B, cudaMemcpyDeviceToDevice, stream));
    if (Q2) MOFEM_CUDA_TRY(cudaMemcpy2DAsync(Q2, w, h->Q2_64, lw, w, q, cudaMemcpyDeviceToDevice, stream));
    if (lambda) MOFEM_CUDA_TRY(cudaMemcpy2DAsync(lambda, w, h->lam64, lw, w, B, cudaMemcpyDeviceToDevice, stream));
    if (mu) MOFEM_CUDA_TRY(cudaMemcpyAsync(mu, h->mu64, w, cudaMemcpyDeviceToDevice, stream));
    if (divisor_product) *divisor_product = h->div_product;
    return MOFEM_OK;
}

mofem_status mofem_destroy(mofem_handle h) {
    if (!h) return MOFEM_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    mofem_free_extra(h);
    mofem_free(h);
    delete h;
    return MOFEM_OK;
}

}  // extern "C"
