// BLAS-1 kernels of the device-resident MO-PCG (Sec. 5, Eq.
// laplace_xnormal_pcg_iteration with the standard PCG recurrences):
//   U += alpha Q,  R -= alpha L(Q), ||R||^2, <R_new, Z_old>        (k_update)
//   <R, Z> and beta after the FP64 preconditioner                  (k_dot)
//   start of an inner solve                                        (k_init)
// plus the small helpers of setup and refinement (conversions, transposes,
// Hadamard divide of the FP64 preconditioner, FP64 correction, IMEX RHS).
//
// Scalars without host round trips: each reducing kernel writes one FP64
// partial per CTA; the last CTA of each instance (atomic ticket after a
// __threadfence) sums that instance's partials in a fixed order and updates
// the instance's PcgScalars (alpha, convergence flags, beta), so results are
// bitwise reproducible and no separate control kernel is needed.  The last CTA
// of the whole update launch sets the CUDA-graph WHILE condition.
//
// Internal q x q matrices use a padded leading dimension ld (multiple of 64)
// whose padding columns stay zero, so the elementwise kernels stream them as
// flat arrays of 16-byte vectors.
#include "internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <type_traits>

namespace {

constexpr int UPD_THREADS = 256;
constexpr int UPD_EVEN_MINB = 3;   // resident CTAs of the even-phase update (registers for 3 x 256 threads)

// RMS of the residual operand in the FP16 preconditioner GEMMs.  The largest
// spectral coefficient of a smooth residual, (Q1^T R Q2)_00, is about q^2 RMS(R)
// (eigenvector entries are O(1) under the mass normalisation); with RMS 2e-3
// the stored intermediates X1^T (~2e-3 q), W^T = T2/(lam+mu) (~1e-4 q^2) and
// Y (~1.5e-4 q^2) stay far below the FP16 maximum 65504 for q up to ~8000,
// while R itself stays in the normal FP16 range down to 3% of its RMS.
constexpr double FP16_RMS = 2e-3;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order sum of n partials by one warp, read through L2 (written by other SMs).
__device__ __forceinline__ double warp_sum_partials(const double* p, int n) {
    double s = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) s += __ldcg(p + i);
    return warp_sum(s);
}

// Block-wide fixed-order sum of one double per thread; result valid in thread 0.
template <int NTH>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NTH / 32; ++w) s += sh[w];
    }
    __syncthreads();
    return s;
}

struct UpdArgs {
    void* U;             // iterate: T (FP64 form) or the hi part of the double-float correction (mixed)
    void* Ulo;           // lo part (mixed form)
    void* R; const void* Q; const void* LQ; const void* Zold; void* Rop;
    const void* Qprev;   // lazy mode: the previous iteration's direction (the other ping-pong buffer)
    int lazy;            // mixed form: add alpha Q to the correction every second iteration, two at a time
    int lazy_phase;      // timing only (no scalar state): force the even (0) or odd (1) form; -1 otherwise
    long long bs;        // batch stride (elements) = q * ld
    long long nvec;      // 16-byte vectors per instance
    double* rr_part; double* rzo_part; int n_upd;
    PcgScalars* sc;
    unsigned* counter;   // [batch] per-instance CTA tickets
    unsigned* gcounter;  // tickets of the whole launch (graph conditional)
    int use_sc, flex, max_iter, fixed;
    double count;        // q * q (unit-RMS scale of the FP16 operand copy)
    cudaGraphConditionalHandle cond;
    int has_cond;
};

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ void axpy_v(float4& u, const float4& q, float a) {
    u.x = fmaf(a, q.x, u.x); u.y = fmaf(a, q.y, u.y); u.z = fmaf(a, q.z, u.z); u.w = fmaf(a, q.w, u.w);
}
__device__ __forceinline__ void axpy_v(double2& u, const double2& q, double a) {
    u.x = fma(a, q.x, u.x); u.y = fma(a, q.y, u.y);
}

__device__ __forceinline__ uint2 pack_f16x4(const float4& r, float sc) {
    __half2 lo = __floats2half2_rn(r.x * sc, r.y * sc);
    __half2 hi = __floats2half2_rn(r.z * sc, r.w * sc);
    uint2 pk;
    pk.x = *reinterpret_cast<unsigned*>(&lo);
    pk.y = *reinterpret_cast<unsigned*>(&hi);
    return pk;
}

__device__ __forceinline__ uint2 pack_bf16x4(const float4& r) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(r.x, r.y);
    __nv_bfloat162 hi = __floats2bfloat162_rn(r.z, r.w);
    uint2 pk;
    pk.x = *reinterpret_cast<unsigned*>(&lo);
    pk.y = *reinterpret_cast<unsigned*>(&hi);
    return pk;
}

// Iterate storage.  FP64 form: U in FP64.  Mixed form: the inner correction is
// accumulated as a double-float pair (hi, lo) of FP32 arrays with error-free
// transformations (exact product alpha*q via FMA, TwoSum, renormalisation), so
// its precision (~2^-48) never limits the refinement, while all arithmetic stays
// on the FP32 pipes (FP64 throughput on this GPU is a small fraction of FP32).
struct DF { float4 h, l; };

__device__ __forceinline__ void df_add_prod(float& h, float& l, float a, float q) {
    const float p = a * q;
    const float e = fmaf(a, q, -p);          // a*q = p + e exactly
    const float s = h + p;
    const float v = s - h;
    float t = (h - (s - v)) + (p - v);       // TwoSum(h, p) error
    t += l + e;
    h = s + t;                               // renormalise
    l = t - (h - s);
}

template <typename T, bool MIXED>
struct UVec;
template <typename T>
struct UVec<T, false> {   // plain iterate in T
    using V = typename Vec<T>::type;
    struct Val { V a; };
    V* p;
    __device__ __forceinline__ Val load(long long i) const { return Val{p[i]}; }
    __device__ __forceinline__ void axpy_store(long long i, Val u, const V& q, T a) {
        axpy_v(u.a, q, a);
        p[i] = u.a;
    }
};
template <>
struct UVec<float, true> {   // double-float correction
    struct Val { float4 h, l; };
    float4* ph;
    float4* pl;
    __device__ __forceinline__ Val load(long long i) const { return Val{ph[i], pl[i]}; }
    __device__ __forceinline__ void axpy_store(long long i, Val u, const float4& q, float a) {
        df_add_prod(u.h.x, u.l.x, a, q.x);
        df_add_prod(u.h.y, u.l.y, a, q.y);
        df_add_prod(u.h.z, u.l.z, a, q.z);
        df_add_prod(u.h.w, u.l.w, a, q.w);
        ph[i] = u.h;
        pl[i] = u.l;
    }
};

// u += a1 q1 + a2 q2 on a double-float pair (two exact products, TwoSum each)
__device__ __forceinline__ void df_axpy2(DF& u, const float4& q1, float a1, const float4& q2, float a2) {
    df_add_prod(u.h.x, u.l.x, a1, q1.x); df_add_prod(u.h.x, u.l.x, a2, q2.x);
    df_add_prod(u.h.y, u.l.y, a1, q1.y); df_add_prod(u.h.y, u.l.y, a2, q2.y);
    df_add_prod(u.h.z, u.l.z, a1, q1.z); df_add_prod(u.h.z, u.l.z, a2, q2.z);
    df_add_prod(u.h.w, u.l.w, a1, q1.w); df_add_prod(u.h.w, u.l.w, a2, q2.w);
}

__device__ __forceinline__ float dot32(const float4& a, const float4& b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ double dot32(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }

// ROP: 0 = no operand copy, 1 = BF16 copy of R for the tensor-core GEMM,
// 2 = FP16 copy of R scaled to unit RMS with the previous ||R|| (the scale is
// recorded in the scalar state and undone by the last GEMM).
// alpha is read from the scalar state (set by the apply kernel's last CTA).
// Dot products: working precision within a thread (a few dozen terms), FP64
// across threads and CTAs (fixed order).
// PH: the lazy phase fixed at compile time (0 even, 1 odd; the iteration graphs hold an even
// and an odd iteration), or -1 to take it from the scalar state.  The even form keeps no
// registers for the correction of U and runs at a higher occupancy.
template <typename T, bool MIXED, int ROP, int PH>
__global__ void __launch_bounds__(UPD_THREADS, PH == 0 ? UPD_EVEN_MINB : 2) k_update(UpdArgs g) {
    static_assert(PH < 0 || MIXED, "a fixed lazy phase belongs to the mixed form");
    constexpr bool HAS_EVEN = PH != 1, HAS_ODD = PH != 0;
    using V = typename Vec<T>::type;
    static_assert(ROP == 0 || Vec<T>::W == 4, "operand copies are produced by the FP32 update only");
    __shared__ double sh[UPD_THREADS / 32];
    __shared__ int last_s, glast_s;
    const int inst = blockIdx.y;
    PcgScalars* sc = g.sc + inst;
    const bool active = !g.use_sc || sc->active;
    if (active) {
        const T alpha = g.use_sc ? (T)sc->alpha : (T)0.5;
        double rs = 1.0;   // FP16 operand scale from the residual norm before this update
        if constexpr (ROP == 2) {
            const double rr_prev = g.use_sc ? sc->rr : g.count;
            rs = rr_prev > 0.0 ? FP16_RMS * sqrt(g.count / rr_prev) : 1.0;
            if (!(rs < 1e30)) rs = 1.0;
        }
        const float rsf = (float)rs;
        UVec<T, MIXED> U;
        if constexpr (MIXED) {
            U.ph = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.U) + (size_t)inst * g.bs);
            U.pl = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.Ulo) + (size_t)inst * g.bs);
        } else {
            U.p = reinterpret_cast<V*>(reinterpret_cast<T*>(g.U) + (size_t)inst * g.bs);
        }
        V* R = reinterpret_cast<V*>(reinterpret_cast<T*>(g.R) + (size_t)inst * g.bs);
        const V* Q = reinterpret_cast<const V*>(reinterpret_cast<const T*>(g.Q) + (size_t)inst * g.bs);
        const V* LQ = reinterpret_cast<const V*>(reinterpret_cast<const T*>(g.LQ) + (size_t)inst * g.bs);
        const V* Zo = reinterpret_cast<const V*>(reinterpret_cast<const T*>(g.Zold) + (size_t)inst * g.bs);
        uint2* Rb = nullptr;
        if constexpr (ROP != 0)
            Rb = reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(g.Rop) + (size_t)inst * g.bs);
        T rrt = (T)0, rzt = (T)0;
        const long long stride = (long long)gridDim.x * blockDim.x;
        constexpr int UNR = 4;   // independent 16-byte loads in flight per thread and array
        long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        // Lazy correction (mixed form): an even iteration only updates R and leaves
        // alpha Q pending; the odd one adds alpha_prev Q_prev + alpha Q in one pass.
        const bool lazy = PH >= 0 || (MIXED && g.lazy && (g.use_sc || g.lazy_phase >= 0));
        const bool pair = PH >= 0 ? PH == 1 : lazy && (g.lazy_phase >= 0 ? g.lazy_phase == 1 : (sc->iters & 1) != 0);
        if constexpr (MIXED) {
            if (lazy) {
                const float4* Qp4 = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(g.Qprev) +
                                                                    (size_t)inst * g.bs);
                const float ap = pair ? (g.use_sc ? (float)sc->alpha_pend : 0.25f) : 0.f;
                auto rbody = [&](long long i, float4 r, const float4& lq, const float4& zo) {
                    axpy_v(r, lq, -alpha);
                    R[i] = r;
                    rrt += dot32(r, r);
                    if (g.flex) rzt += dot32(r, zo);
                    if constexpr (ROP == 1) Rb[i] = pack_bf16x4(r);
                    if constexpr (ROP == 2) Rb[i] = pack_f16x4(r, rsf);
                };
                // batches of independent 16-byte loads in flight per thread (memory-level parallelism)
                if (!pair) {
                  if constexpr (HAS_EVEN) {
                    constexpr int UE = 4;
                    for (; i0 + (UE - 1) * stride < g.nvec; i0 += UE * stride) {
                        float4 r[UE], lq[UE], zo[UE];
#pragma unroll
                        for (int k = 0; k < UE; ++k) {
                            const long long i = i0 + k * stride;
                            r[k] = R[i];
                            lq[k] = LQ[i];
                            zo[k] = g.flex ? Zo[i] : lq[k];
                        }
#pragma unroll
                        for (int k = 0; k < UE; ++k) rbody(i0 + k * stride, r[k], lq[k], zo[k]);
                    }
                  }
                } else {
                  if constexpr (HAS_ODD) {
                    constexpr int UO = 2;
                    for (; i0 + (UO - 1) * stride < g.nvec; i0 += UO * stride) {
                        float4 r[UO], lq[UO], zo[UO], qp[UO], qc[UO];
                        DF u[UO];
#pragma unroll
                        for (int k = 0; k < UO; ++k) {
                            const long long i = i0 + k * stride;
                            r[k] = R[i];
                            lq[k] = LQ[i];
                            zo[k] = g.flex ? Zo[i] : lq[k];
                            u[k] = DF{U.ph[i], U.pl[i]};
                            qp[k] = Qp4[i];
                            qc[k] = Q[i];
                        }
#pragma unroll
                        for (int k = 0; k < UO; ++k) {
                            const long long i = i0 + k * stride;
                            df_axpy2(u[k], qp[k], ap, qc[k], alpha);
                            U.ph[i] = u[k].h;
                            U.pl[i] = u[k].l;
                            rbody(i, r[k], lq[k], zo[k]);
                        }
                    }
                  }
                }
                for (; i0 < g.nvec; i0 += stride) {
                    float4 r = R[i0];
                    const float4 lq = LQ[i0];
                    const float4 zo = g.flex ? Zo[i0] : lq;
                    if (HAS_ODD && pair) {
                        DF u{U.ph[i0], U.pl[i0]};
                        df_axpy2(u, Qp4[i0], ap, Q[i0], alpha);
                        U.ph[i0] = u.h;
                        U.pl[i0] = u.l;
                    }
                    rbody(i0, r, lq, zo);
                }
            }
        }
        if constexpr (PH < 0) if (!lazy) {
        using UV = typename UVec<T, MIXED>::Val;
        auto body = [&](long long i, UV u, V r, const V& qv, const V& lq, const V& zo) {
            U.axpy_store(i, u, qv, alpha);
            axpy_v(r, lq, -alpha);
            R[i] = r;
            rrt += dot32(r, r);
            if (g.flex) rzt += dot32(r, zo);
            if constexpr (ROP == 1) Rb[i] = pack_bf16x4(r);
            if constexpr (ROP == 2) Rb[i] = pack_f16x4(r, rsf);
        };
        for (; i0 + (UNR - 1) * stride < g.nvec; i0 += UNR * stride) {
            UV u[UNR];
            V r[UNR], qv[UNR], lq[UNR], zo[UNR];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const long long i = i0 + k * stride;
                u[k] = U.load(i);
                r[k] = R[i];
                qv[k] = Q[i];
                lq[k] = LQ[i];
                zo[k] = g.flex ? Zo[i] : qv[k];
            }
#pragma unroll
            for (int k = 0; k < UNR; ++k) body(i0 + k * stride, u[k], r[k], qv[k], lq[k], zo[k]);
        }
        for (; i0 < g.nvec; i0 += stride) body(i0, U.load(i0), R[i0], Q[i0], LQ[i0], g.flex ? Zo[i0] : Q[i0]);
        }
        const double rr = (double)rrt, rzo = (double)rzt;
        const double s1 = block_sum<UPD_THREADS>(rr, sh);
        const double s2 = block_sum<UPD_THREADS>(rzo, sh);
        if (threadIdx.x == 0) {
            g.rr_part[(size_t)inst * g.n_upd + blockIdx.x] = s1;
            g.rzo_part[(size_t)inst * g.n_upd + blockIdx.x] = s2;
            __threadfence();
            const unsigned t = atomicAdd(g.counter + inst, 1u);
            last_s = (t == gridDim.x - 1) ? 1 : 0;
        }
        __syncthreads();
        if (last_s && threadIdx.x < 32) {
            __threadfence();
            const double rrs = warp_sum_partials(g.rr_part + (size_t)inst * g.n_upd, g.n_upd);
            const double rzs = warp_sum_partials(g.rzo_part + (size_t)inst * g.n_upd, g.n_upd);
            if (threadIdx.x == 0) {
                g.counter[inst] = 0;
                if (g.use_sc) {
                    const int it = sc->iters + 1;
                    sc->iters = it;
                    sc->rr = rrs;
                    if (g.flex) sc->rzo = rzs;   // else set by the apply kernel
                    if (lazy) sc->alpha_pend = pair ? 0.0 : (double)alpha;
                    if (ROP == 2) sc->rscale = rs;
                    int act = 1;
                    if (!isfinite(rrs)) {
                        sc->status |= DEV_ERR_NONFINITE;
                        act = 0;
                    } else if (!g.fixed && rrs <= sc->tol2) {
                        act = 0;
                    } else if (it >= g.max_iter) {
                        act = 0;
                    }
                    sc->active = act;
                }
            }
        }
    }
    // graph conditional: the last CTA of the launch sets "some instance active"
    if (g.has_cond) {
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned t = atomicAdd(g.gcounter, 1u);
            glast_s = (t == gridDim.x * gridDim.y - 1) ? 1 : 0;
        }
        __syncthreads();
        if (glast_s && threadIdx.x == 0) {
            __threadfence();
            int any = 0;
            for (unsigned i = 0; i < gridDim.y; ++i) any |= __ldcg(&g.sc[i].active);
            *g.gcounter = 0;
            cudaGraphSetConditional(g.cond, any ? 1u : 0u);
        }
    }
}

// Start of an inner solve: rr0 = ||R0||^2, stop threshold tol2 = rtol^2 * ref2
// (ref2 = rr0 when no reference is given), counters.  One warp per instance.
struct InitArgs {
    PcgScalars* sc;
    const double* rr; int n_rr;   // partials of ||R0||^2
    const double* ref2;           // [batch] or nullptr
    int batch;
    double rtol;
    double count;                 // q * q
};

__global__ void k_init(InitArgs g) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int inst = warp; inst < g.batch; inst += nw) {
        double rr = warp_sum_partials(g.rr + (size_t)inst * g.n_rr, g.n_rr);
        if (lane == 0) {
            PcgScalars* s = g.sc + inst;
            const double ref = g.ref2 ? g.ref2[inst] : rr;
            s->rr0 = rr;
            s->rr = rr;
            s->tol2 = g.rtol * g.rtol * ref;
            s->iters = 0;
            s->alpha = 0.0;
            s->beta = 0.0;
            s->rz = 1.0;
            s->rzo = 0.0;
            s->rscale = (rr > 0.0 && isfinite(rr)) ? FP16_RMS * sqrt(g.count / rr) : 1.0;
            s->alpha_pend = 0.0;
            s->status = isfinite(rr) ? 0 : DEV_ERR_NONFINITE;
            s->active = (rr > s->tol2 && isfinite(rr)) ? 1 : 0;
        }
    }
}

// IMEX right-hand side in nodal form: Fbar = gam * (cu pad(U_n) + tau F_n), n x n
// per instance; U_n is q x q (boundary nodes zero under Dirichlet); cu = 1 - tau r
// for an explicit linear reaction -r u.
__global__ void k_imex_rhs(const double* Un, const double* Fn, double* Fbar, int n, int q, int off, double gam,
                           double tau, double cu) {
    const int inst = blockIdx.z, r = blockIdx.y;
    const double* fn = Fn + (size_t)inst * n * n + (size_t)r * n;
    double* fb = Fbar + (size_t)inst * n * n + (size_t)r * n;
    const int ur = r - off;
    for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < n; cc += gridDim.x * blockDim.x) {
        const int uc = cc - off;
        double u = 0.0;
        if (ur >= 0 && ur < q && uc >= 0 && uc < q) u = Un[(size_t)inst * q * q + (size_t)ur * q + uc];
        fb[cc] = gam * (cu * u + tau * fn[cc]);
    }
}

// Dot-product partials <A, B> over a flat [batch][n] range.  With `sc`, the
// last CTA of each instance sums them in a fixed order and performs the
// preconditioner finalisation of the PCG: rz_new = <R, Z>,
// beta = (rz_new - flex <R_new, Z_old>) / rz_old.
template <typename T>
__global__ void __launch_bounds__(UPD_THREADS) k_dot(const T* A, const T* B, long long bs, long long n,
                                                    double* part, int nblk, PcgScalars* sc, unsigned* counter,
                                                    int flex) {
    __shared__ double sh[UPD_THREADS / 32];
    __shared__ int last_s;
    const int inst = blockIdx.y;
    if (sc && !sc[inst].active) return;
    A += (size_t)inst * bs;
    B += (size_t)inst * bs;
    double acc = 0.0;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 within a thread (a few dozen terms, 16-byte loads where aligned), FP64 across
        // threads: a conversion per element would run on the FP64 pipe (a small fraction of
        // the FP32 rate on this GPU)
        float a32 = 0.f;
        const bool vec = (n % 4) == 0 && (bs % 4) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0 &&
                         (reinterpret_cast<uintptr_t>(B) % 16) == 0;
        if (vec) {
            const float4* A4 = reinterpret_cast<const float4*>(A);
            const float4* B4 = reinterpret_cast<const float4*>(B);
            for (long long i = t0; i < n / 4; i += stride) {
                const float4 a = A4[i], b = B4[i];
                a32 = fmaf(a.x, b.x, a32);
                a32 = fmaf(a.y, b.y, a32);
                a32 = fmaf(a.z, b.z, a32);
                a32 = fmaf(a.w, b.w, a32);
            }
        } else {
            for (long long i = t0; i < n; i += stride) a32 = fmaf(A[i], B[i], a32);
        }
        acc = (double)a32;
    } else {
        for (long long i = t0; i < n; i += stride) acc += (double)A[i] * (double)B[i];
    }
    double s = block_sum<UPD_THREADS>(acc, sh);
    if (threadIdx.x == 0) {
        part[(size_t)inst * nblk + blockIdx.x] = s;
        if (sc) {
            __threadfence();
            const unsigned t = atomicAdd(counter + inst, 1u);
            last_s = (t == (unsigned)nblk - 1) ? 1 : 0;
        }
    }
    if (!sc) return;
    __syncthreads();
    if (last_s && threadIdx.x < 32) {
        __threadfence();
        const double rz = warp_sum_partials(part + (size_t)inst * nblk, nblk);
        if (threadIdx.x == 0) {
            counter[inst] = 0;
            PcgScalars* p = sc + inst;
            double beta = (rz - (flex ? p->rzo : 0.0)) / p->rz;
            if (!isfinite(beta)) beta = 0.0;
            p->beta = beta;
            p->rz = rz;
        }
    }
}

template <typename S, typename D>
__global__ void k_convert(const S* src, long long s_bs, int s_ld, D* dst, long long d_bs, int d_ld, int rows, int cols) {
    const int inst = blockIdx.z;
    const int r = blockIdx.y;
    src += (size_t)inst * s_bs + (size_t)r * s_ld;
    dst += (size_t)inst * d_bs + (size_t)r * d_ld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        if constexpr (std::is_same<D, __nv_bfloat16>::value) dst[c] = __float2bfloat16_rn((float)src[c]);
        else if constexpr (std::is_same<D, __half>::value) dst[c] = __float2half_rn((float)src[c]);
        else dst[c] = (D)src[c];
    }
}

__global__ void k_convert_scaled_f16(const float* src, long long s_bs, int s_ld, __half* dst, long long d_bs, int d_ld,
                                     int cols, const PcgScalars* sc) {
    const int inst = blockIdx.z, r = blockIdx.y;
    const float s = (float)sc[inst].rscale;
    src += (size_t)inst * s_bs + (size_t)r * s_ld;
    dst += (size_t)inst * d_bs + (size_t)r * d_ld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
        dst[c] = __float2half_rn(src[c] * s);
}

__global__ void k_set_rscale(PcgScalars* sc, const double* part, int nper, int batch, double count) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int inst = warp; inst < batch; inst += nw) {
        const double ss = warp_sum_partials(part + (size_t)inst * nper, nper);
        if (lane == 0) sc[inst].rscale = (ss > 0.0 && isfinite(ss)) ? FP16_RMS * sqrt(count / ss) : 1.0;
    }
}

__global__ void k_transpose64(const double* src, long long s_bs, double* dst, long long d_bs, int n, int s_ld, int d_ld) {
    __shared__ double tile[32][33];
    const int inst = blockIdx.z;
    src += (size_t)inst * s_bs;
    dst += (size_t)inst * d_bs;
    int x = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int y = y0 + j;
        if (x < n && y < n) tile[j][threadIdx.x] = src[(size_t)y * s_ld + x];
    }
    __syncthreads();
    x = blockIdx.y * 32 + threadIdx.x;
    y0 = blockIdx.x * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int y = y0 + j;
        if (x < n && y < n) dst[(size_t)y * d_ld + x] = tile[threadIdx.x][j];
    }
}

__global__ void k_hadamard_div64(double* W, long long bs, int ld, int q, const double* lam, long long lam_bs,
                                 const double* mu, int product) {
    const int inst = blockIdx.z, i = blockIdx.y;
    const double li = lam[(size_t)inst * lam_bs + i];
    double* row = W + (size_t)inst * bs + (size_t)i * ld;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < q; j += gridDim.x * blockDim.x)
        row[j] /= product ? li * mu[j] : li + mu[j];
}

// U64 += d with d = hi + lo (+ alpha_pend Q_pend, the last even iteration's term
// when the correction is accumulated lazily) at the end of an inner solve of the
// mixed form; the pair is cleared before the next inner solve starts.  d is formed
// in FP64 and added with one rounding.  With `write_d` the pair is overwritten by
// the step actually taken, d - err with err = (U + d) - fl(U + d) exact by TwoSum,
// as a double-float (hi, lo): a residual update R -= L(hi + lo) then tracks
// B - L(U) of the stored iterate, up to the pair's rounding of that step (2^-48 of it).
// 16-byte vectors: n % 4 == 0.  (Mode 2, a step from U = 0, is k_fold_zero.)
__device__ __forceinline__ double fold_one(double u, float& h, float& l, double ap, float q, int write_d) {
    double d = (double)h + (double)l;
    if (ap != 0.0) d = fma(ap, (double)q, d);
    const double s = u + d;
    if (write_d) {
        // the step taken, s - u: exact when |d| <= |u| (Fast2Sum), else d minus the TwoSum error
        double taken = s - u;
        if (!(fabs(d) <= fabs(u))) {
            const double v = s - u;
            taken = d - ((u - (s - v)) + (d - v));
        }
        h = (float)taken;
        l = (float)(taken - (double)h);
    }
    return s;
}

__global__ void k_fold_df(double* U, long long bs, float* hi, float* lo, long long n, const PcgScalars* sc,
                          const float* Qpend, int write_d) {
    const int inst = blockIdx.y;
    const double ap = sc ? sc[inst].alpha_pend : 0.0;
    double2* U2 = reinterpret_cast<double2*>(U + (size_t)inst * bs);
    float4* h4 = reinterpret_cast<float4*>(hi + (size_t)inst * bs);
    float4* l4 = reinterpret_cast<float4*>(lo + (size_t)inst * bs);
    const float4* q4 = reinterpret_cast<const float4*>(Qpend + (size_t)inst * bs);
    const long long nv = n / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        float4 h = h4[i], l = l4[i];
        const float4 q = ap != 0.0 ? q4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        double2 a = U2[2 * i], b = U2[2 * i + 1];
        a.x = fold_one(a.x, h.x, l.x, ap, q.x, write_d);
        a.y = fold_one(a.y, h.y, l.y, ap, q.y, write_d);
        b.x = fold_one(b.x, h.z, l.z, ap, q.z, write_d);
        b.y = fold_one(b.y, h.w, l.w, ap, q.w, write_d);
        U2[2 * i] = a;
        U2[2 * i + 1] = b;
        if (write_d) {
            h4[i] = h;
            l4[i] = l;
        }
    }
}

// The fold of a step from U = 0 (mode 2 of launch_fold_df): the step d = hi + lo
// (+ alpha_pend Q_pend) formed in double-float arithmetic on the FP32 pipes, its low
// part rounded onto the FP64 grid of its high part (multiples of 2^(e_hi - 52)), so that
// hi + lo is exact in FP64.  The iterate becomes that sum and the pair is rewritten as
// the step itself: one FP64 add and two conversions per element (this GPU's FP64 rate
// is a small fraction of its FP32 rate).  |hi| < 2^-97 keeps hi alone.
__device__ __forceinline__ double fold_zero_one(float& h, float& l, float aph, float apl, float q, bool pend) {
    float s, lo;
    {   // the accumulated pair may be unnormalised: TwoSum first
        s = h + l;
        const float v = s - h;
        lo = (h - (s - v)) + (l - v);
    }
    if (pend) {   // + (aph + apl) q: exact high product, its error and the low product into lo
        const float p = aph * q;
        float e = fmaf(aph, q, -p);
        e = fmaf(apl, q, e);
        const float t = s + p, v = t - s;
        const float r = (s - (t - v)) + (p - v);
        s = t;
        lo = (lo + e) + r;
    }
    const float H = s + lo, v = H - s;
    float L = (s - (H - v)) + (lo - v);
    if (H != 0.f) {
        const int eh = ilogbf(H);
        L = eh >= -97 ? ldexpf(rintf(ldexpf(L, 52 - eh)), eh - 52) : 0.f;
    }
    h = H;
    l = L;
    return (double)H + (double)L;
}

__global__ void k_fold_zero(double* U, long long bs, float* hi, float* lo, long long n, const PcgScalars* sc,
                            const float* Qpend) {
    const int inst = blockIdx.y;
    const double ap = sc ? sc[inst].alpha_pend : 0.0;
    const float aph = (float)ap, apl = (float)(ap - (double)aph);
    const bool pend = ap != 0.0;
    double2* U2 = reinterpret_cast<double2*>(U + (size_t)inst * bs);
    float4* h4 = reinterpret_cast<float4*>(hi + (size_t)inst * bs);
    float4* l4 = reinterpret_cast<float4*>(lo + (size_t)inst * bs);
    const float4* q4 = reinterpret_cast<const float4*>(Qpend + (size_t)inst * bs);
    const long long nv = n / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
        float4 h = h4[i], l = l4[i];
        const float4 q = pend ? q4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        double2 a, b;
        a.x = fold_zero_one(h.x, l.x, aph, apl, q.x, pend);
        a.y = fold_zero_one(h.y, l.y, aph, apl, q.y, pend);
        b.x = fold_zero_one(h.z, l.z, aph, apl, q.z, pend);
        b.y = fold_zero_one(h.w, l.w, aph, apl, q.w, pend);
        U2[2 * i] = a;
        U2[2 * i + 1] = b;
        h4[i] = h;
        l4[i] = l;
    }
}

__global__ void k_axpy_into64(double* U, long long u_bs, int u_ld, const float* d, long long d_bs, int d_ld, int q) {
    const int inst = blockIdx.z, r = blockIdx.y;
    double* u = U + (size_t)inst * u_bs + (size_t)r * u_ld;
    const float* dv = d + (size_t)inst * d_bs + (size_t)r * d_ld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q; c += gridDim.x * blockDim.x) u[c] += (double)dv[c];
}

// dst = s * src over rows x cols (FP64, own leading dimensions).
__global__ void k_scale_copy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld,
                               int cols, double s) {
    const int inst = blockIdx.z, r = blockIdx.y;
    const double* a = src + (size_t)inst * s_bs + (size_t)r * s_ld;
    double* b = dst + (size_t)inst * d_bs + (size_t)r * d_ld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) b[c] = s * a[c];
}

// Graph conditional of the heterogeneous lockstep loop: 1 while any instance of any group
// is active.  One block.
__global__ void k_set_cond_any(PcgScalars* const* scs, const int* batch, int ngroups, cudaGraphConditionalHandle h) {
    __shared__ int any_s;
    if (threadIdx.x == 0) any_s = 0;
    __syncthreads();
    int any = 0;
    for (int gi = 0; gi < ngroups; ++gi)
        for (int i = threadIdx.x; i < batch[gi]; i += blockDim.x) any |= __ldcg(&scs[gi][i].active);
    if (any) atomicOr(&any_s, 1);
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any_s ? 1u : 0u);
}

// dst += a * src, rows x cols per instance (FP64).
__global__ void k_axpy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld, int cols,
                         double a) {
    const int inst = blockIdx.z, r = blockIdx.y;
    const double* x = src + (size_t)inst * s_bs + (size_t)r * s_ld;
    double* y = dst + (size_t)inst * d_bs + (size_t)r * d_ld;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) y[c] += a * x[c];
}

}  // namespace

mofem_status launch_set_cond_any(PcgScalars* const* scs, const int* batch, int ngroups, cudaGraphConditionalHandle h,
                                 cudaStream_t st) {
    k_set_cond_any<<<1, 128, 0, st>>>(scs, batch, ngroups, h);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_axpy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld, int rows,
                           int cols, int batch, double a, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || batch <= 0) return MOFEM_OK;
    dim3 grid((cols + 255) / 256, rows, batch);
    k_axpy64<<<grid, 256, 0, st>>>(src, s_bs, s_ld, dst, d_bs, d_ld, cols, a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

// ---------------------------------------------------------------------------
mofem_status launch_pcg_update(const mofem_ctx* c, bool fp64, void* U, void* Ulo, void* R, const void* Q,
                               const void* LQ, const void* Zold, void* Rop, int rop_kind, int flex, int max_iter,
                               bool fixed, const cudaGraphConditionalHandle* cond, cudaStream_t st, bool use_scalars,
                               const void* Qprev, int lazy_phase) {
    UpdArgs g;
    g.U = U; g.Ulo = Ulo; g.R = R; g.Q = Q; g.LQ = LQ; g.Zold = Zold; g.Rop = Rop;
    g.Qprev = Qprev;
    g.lazy = (!fp64 && Qprev) ? 1 : 0;
    g.lazy_phase = lazy_phase;
    g.bs = (long long)c->q * c->ld;
    g.nvec = g.bs / (fp64 ? 2 : 4);
    g.rr_part = c->part.rr; g.rzo_part = c->part.rzo; g.n_upd = c->part.n_upd;
    g.sc = c->d_sc;
    g.counter = c->d_ctr + 1 * c->batch;
    g.gcounter = c->d_ctr + 4 * c->batch;
    g.use_sc = use_scalars ? 1 : 0;
    g.flex = flex;
    g.max_iter = max_iter;
    g.fixed = fixed ? 1 : 0;
    g.has_cond = (cond && use_scalars) ? 1 : 0;
    g.cond = cond ? *cond : 0;
    dim3 grid(c->part.n_upd, c->batch);
    g.count = (double)c->q * c->q;
    void (*kern)(UpdArgs) = nullptr;
    int wave_slot = -1;
    if (fp64) kern = k_update<double, false, 0, -1>;
    else if (g.lazy && lazy_phase >= 0) {   // the phase is known when the iteration is recorded
        const int rk = rop_kind == 1 ? 1 : (rop_kind == 2 ? 2 : 0);
        wave_slot = rk * 2 + (lazy_phase ? 1 : 0);
        if (lazy_phase == 0)
            kern = rk == 1 ? k_update<float, true, 1, 0> : (rk == 2 ? k_update<float, true, 2, 0> : k_update<float, true, 0, 0>);
        else
            kern = rk == 1 ? k_update<float, true, 1, 1> : (rk == 2 ? k_update<float, true, 2, 1> : k_update<float, true, 0, 1>);
    } else {
        kern = rop_kind == 1 ? k_update<float, true, 1, -1>
                             : (rop_kind == 2 ? k_update<float, true, 2, -1> : k_update<float, true, 0, -1>);
    }
    if (wave_slot >= 0) {
        // phase-specialised forms: one wave of resident CTAs over all instances (the partial
        // slots, n_upd per instance, are the upper bound)
        static std::atomic<int> wave[6][MOFEM_MAX_DEV];
        std::atomic<int>& w = wave[wave_slot][dev_slot()];
        int n = w.load(std::memory_order_relaxed);
        if (!n) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, UPD_THREADS, 0) != cudaSuccess || per < 1)
                per = 1;
            n = (sms > 0 ? sms : 1) * per;
            w.store(n, std::memory_order_relaxed);
        }
        const int nx = std::max(1, std::min(c->part.n_upd, n / c->batch));
        grid.x = nx;
        g.n_upd = nx;
    }
    kern<<<grid, UPD_THREADS, 0, st>>>(g);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_pcg_init(const mofem_ctx* c, const double* rr_partials, int n_rr, const double* ref2, double rtol,
                             cudaStream_t st) {
    InitArgs g;
    g.sc = c->d_sc;
    g.rr = rr_partials; g.n_rr = n_rr;
    g.ref2 = ref2;
    g.batch = c->batch;
    g.rtol = rtol;
    g.count = (double)c->q * c->q;
    k_init<<<1, 256, 0, st>>>(g);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_imex_rhs(const double* Un, const double* Fn, double* Fbar, int n, int q, int off, double gam,
                             double tau, double cu, int batch, cudaStream_t st) {
    dim3 grid((n + 255) / 256, n, batch);
    k_imex_rhs<<<grid, 256, 0, st>>>(Un, Fn, Fbar, n, q, off, gam, tau, cu);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_dot_partials(const void* A, const void* B, bool fp64, long long bs, long long n, int batch,
                                 double* part, int nblk, cudaStream_t st, PcgScalars* sc, unsigned* counter, int flex) {
    dim3 grid(nblk, batch);
    if (fp64)
        k_dot<double><<<grid, UPD_THREADS, 0, st>>>((const double*)A, (const double*)B, bs, n, part, nblk, sc, counter,
                                                    flex);
    else
        k_dot<float><<<grid, UPD_THREADS, 0, st>>>((const float*)A, (const float*)B, bs, n, part, nblk, sc, counter,
                                                   flex);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_convert(const void* src, int sk, long long s_bs, int s_ld, void* dst, int dk, long long d_bs,
                            int d_ld, int rows, int cols, int batch, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || batch <= 0) return MOFEM_OK;
    dim3 grid((cols + 255) / 256, rows, batch);
#define CONV(S, D) k_convert<S, D><<<grid, 256, 0, st>>>((const S*)src, s_bs, s_ld, (D*)dst, d_bs, d_ld, rows, cols)
    if (sk == 0 && dk == 0) CONV(float, float);
    else if (sk == 0 && dk == 1) CONV(float, double);
    else if (sk == 0 && dk == 2) CONV(float, __nv_bfloat16);
    else if (sk == 1 && dk == 0) CONV(double, float);
    else if (sk == 1 && dk == 1) CONV(double, double);
    else if (sk == 1 && dk == 2) CONV(double, __nv_bfloat16);
    else if (sk == 0 && dk == 3) CONV(float, __half);
    else if (sk == 1 && dk == 3) CONV(double, __half);
    else return MOFEM_ERR_UNSUPPORTED;
#undef CONV
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_transpose64(const double* src, long long s_bs, double* dst, long long d_bs, int n, int ld,
                                int batch, cudaStream_t st) {
    // src: n x n with leading dimension n (dense); dst: leading dimension ld
    dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
    k_transpose64<<<grid, dim3(32, 8), 0, st>>>(src, s_bs, dst, d_bs, n, n, ld);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_transpose64_ld(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld,
                                   int n, int batch, cudaStream_t st) {
    dim3 grid((n + 31) / 32, (n + 31) / 32, batch);
    k_transpose64<<<grid, dim3(32, 8), 0, st>>>(src, s_bs, dst, d_bs, n, s_ld, d_ld);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_hadamard_div64(double* W, long long bs, int ld, int q, const double* lam, long long lam_bs,
                                   const double* mu, int batch, int product, cudaStream_t st) {
    dim3 grid((q + 255) / 256, q, batch);
    k_hadamard_div64<<<grid, 256, 0, st>>>(W, bs, ld, q, lam, lam_bs, mu, product);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_axpy_into64(double* U64, long long u_bs, int u_ld, const float* dU, long long d_bs, int d_ld,
                                int q, int batch, cudaStream_t st) {
    dim3 grid((q + 255) / 256, q, batch);
    k_axpy_into64<<<grid, 256, 0, st>>>(U64, u_bs, u_ld, dU, d_bs, d_ld, q);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_fold_df(double* U64, float* hi, float* lo, long long bs, int batch, const PcgScalars* sc,
                            const float* Qpend, int write_d, cudaStream_t st) {
    if (bs % 4 != 0) return MOFEM_ERR_INVALID_ARG;   // internal layout: ld is a multiple of 64
    if (write_d < 0 || write_d > 2) return MOFEM_ERR_INVALID_ARG;
    dim3 grid(592, batch);
    if (write_d == 2)   // the iterate is zero before this fold: not read
        k_fold_zero<<<grid, 256, 0, st>>>(U64, bs, hi, lo, bs, sc, Qpend);
    else
        k_fold_df<<<grid, 256, 0, st>>>(U64, bs, hi, lo, bs, sc, Qpend, write_d);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_convert_scaled_f16(const float* src, long long s_bs, int s_ld, void* dst, long long d_bs, int d_ld,
                                       int rows, int cols, int batch, const PcgScalars* sc, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || batch <= 0) return MOFEM_OK;
    dim3 grid((cols + 255) / 256, rows, batch);
    k_convert_scaled_f16<<<grid, 256, 0, st>>>(src, s_bs, s_ld, (__half*)dst, d_bs, d_ld, cols, sc);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_set_rscale(PcgScalars* sc, const double* part, int nper, int batch, double count, cudaStream_t st) {
    k_set_rscale<<<1, 256, 0, st>>>(sc, part, nper, batch, count);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

mofem_status launch_scale_copy64(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld,
                                 int rows, int cols, int batch, double scale, cudaStream_t st) {
    if (rows <= 0 || cols <= 0 || batch <= 0) return MOFEM_OK;
    dim3 grid((cols + 255) / 256, rows, batch);
    k_scale_copy64<<<grid, 256, 0, st>>>(src, s_bs, s_ld, dst, d_bs, d_ld, cols, scale);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}
