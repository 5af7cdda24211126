// DIB reaction-diffusion model (Sec. 7, Eqs. dib_model, dib_kinetics_f,
// dib_kinetics_g): explicit kinetics kernel and the IMEX Euler time loop whose
// diffusion steps are batched MO-PCG solves (the two species are the two
// instances of one handle, with gamma_i = 1/(d_i tau), d_eta = 1, d_theta from
// the parameters).
//
//   f(eta, theta) = A1 (1 - theta) eta - A2 eta^3 - B (theta - alpha)
//   g(eta, theta) = C (1 + k2 eta)(1 - theta)[1 - gamma (1 - theta)]
//                   - D theta (1 + gamma theta)(1 + k3 eta)
//
// One step: F = rho (f, g)(U_n) at every node (homogeneous Neumann: the unknowns
// are all nodes), then (M~ + d_i tau A~) U_{n+1,i} = M~ (U_{n,i} + tau F_i) for
// both species in one batched solve.
#include "internal.h"

#include <cmath>
#include <vector>

namespace {

__global__ void k_dib_kinetics(mofem_dib_params p, double rho, const double* __restrict__ eta,
                               const double* __restrict__ theta, double* __restrict__ f, double* __restrict__ g,
                               long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double e = eta[i], t = theta[i], u = 1.0 - t;
        f[i] = rho * (p.A1 * u * e - p.A2 * e * e * e - p.B * (t - p.alpha));
        g[i] = rho * (p.C * (1.0 + p.k2 * e) * u * (1.0 - p.gamma * u) - p.D * t * (1.0 + p.gamma * t) * (1.0 + p.k3 * e));
    }
}

// ||A - B||_F^2 per block (FP64 partials, summed on the host in a fixed order).
__global__ void k_diff_norm2(const double* __restrict__ a, const double* __restrict__ b, long long n, double* part) {
    __shared__ double sh[8];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = a[i] - b[i];
        s = fma(d, d, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

}  // namespace

mofem_status launch_dib_kinetics(const mofem_dib_params& p, double rho, const double* eta, const double* theta,
                                 double* f, double* g, long long n, cudaStream_t st) {
    if (n <= 0) return MOFEM_OK;
    const long long blocks = (n + 255) / 256;
    k_dib_kinetics<<<(unsigned)(blocks < 1184 ? blocks : 1184), 256, 0, st>>>(p, rho, eta, theta, f, g, n);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

// n_steps of the DIB model on a two-instance handle: U holds [eta; theta], q x q
// each (ld q), updated in place.  incr (host, may be null) receives
// ||eta_{k+1} - eta_k||_F per step.
mofem_status dib_run(mofem_ctx* c, const mofem_dib_params& p, double rho, double tau, int n_steps, double* U,
                     double rtol, mofem_precision prec, double* incr, mofem_solve_info* info, cudaStream_t st) {
    const int q = c->q;
    const long long qq = (long long)q * q;
    constexpr int NB = 256;
    double* buf = nullptr;
    // F (2 x q x q), U_next (2 x q x q), partials
    MOFEM_CUDA_TRY(cudaMallocAsync((void**)&buf, sizeof(double) * (size_t)(4 * qq + NB), st));
    double *F = buf, *Un = buf + 2 * qq, *part = buf + 4 * qq;
    mofem_status s = MOFEM_OK;
    mofem_solve_info acc{};
    std::vector<double> hp(NB);
    for (int k = 0; k < n_steps && s == MOFEM_OK; ++k) {
        s = launch_dib_kinetics(p, rho, U, U + qq, F, F + qq, qq, st);
        mofem_solve_info one{};
        if (s == MOFEM_OK) s = solve_imex(c, 0.0, tau, U, F, Un, rtol, prec, &one, st);
        acc.iterations += one.iterations;
        acc.outer_steps += one.outer_steps;
        acc.kernel_launches += one.kernel_launches + 1;
        acc.ms_total += one.ms_total;
        if (one.rel_residual > acc.rel_residual) acc.rel_residual = one.rel_residual;
        if (s != MOFEM_OK) break;
        if (incr) {
            k_diff_norm2<<<NB, 256, 0, st>>>(Un, U, qq, part);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(hp.data(), part, sizeof(double) * NB, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                s = MOFEM_ERR_CUDA;
                break;
            }
            double t = 0.0;
            for (double v : hp) t += v;
            incr[k] = sqrt(t);
            acc.kernel_launches += 1;
        }
        if (cudaMemcpyAsync(U, Un, sizeof(double) * 2 * qq, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            s = MOFEM_ERR_CUDA;
    }
    cudaFreeAsync(buf, st);
    if (info) {
        acc.status = s;
        acc.batch = c->batch;
        *info = acc;
    }
    return s;
}

// Homogeneous equilibrium f = g = 0 by Newton's method from (0, 1/2), with the
// analytic Jacobian of the kinetics (host, FP64).
mofem_status dib_equilibrium(const mofem_dib_params& p, double* eta, double* theta) {
    double e = 0.0, t = 0.5;
    for (int it = 0; it < 100; ++it) {
        const double u = 1.0 - t, w = 1.0 - p.gamma * u;
        const double f = p.A1 * u * e - p.A2 * e * e * e - p.B * (t - p.alpha);
        const double g = p.C * (1.0 + p.k2 * e) * u * w - p.D * t * (1.0 + p.gamma * t) * (1.0 + p.k3 * e);
        const double fe = p.A1 * u - 3.0 * p.A2 * e * e;
        const double ft = -p.A1 * e - p.B;
        const double ge = p.C * p.k2 * u * w - p.D * t * (1.0 + p.gamma * t) * p.k3;
        // d/dt [u w] = -w + u gamma ;  d/dt [t (1 + gamma t)] = 1 + 2 gamma t
        const double gt = p.C * (1.0 + p.k2 * e) * (-w + u * p.gamma) - p.D * (1.0 + 2.0 * p.gamma * t) * (1.0 + p.k3 * e);
        const double det = fe * gt - ft * ge;
        if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return MOFEM_ERR_NONFINITE;
        const double de = (f * gt - ft * g) / det, dt = (fe * g - ge * f) / det;
        e -= de;
        t -= dt;
        if (std::fabs(de) + std::fabs(dt) <= 1e-15 * (1.0 + std::fabs(e) + std::fabs(t))) break;
    }
    if (!std::isfinite(e) || !std::isfinite(t)) return MOFEM_ERR_NONFINITE;
    *eta = e;
    *theta = t;
    return MOFEM_OK;
}
