// Banded multiterm operator apply  Y = sum_i S_i X T_i^T  (Sec. 5, operator L~;
// Eq. laplace_cap-shaped-domain_sylvester), the operator of every MO-PCG
// iteration.
//
// Data: X, Y row-major (rows = s-nodes a, columns = t-nodes b).  S_i and T_i are
// banded with half-bandwidth K (the element degree), stored diagonal-major:
// tab[i][j][r] = M_i[r][r + off + j - K] (0 outside the matrix).  Tables used in
// difference form (all T tables, the S tables of stiffness- and convection-like
// terms) hold the row sum in the diagonal slot j = K instead of the diagonal.
//
// Difference form: (A x)_r = rowsum_r x_r + sum_{j != K} A_rj (x_{r+j-K} - x_r).
// It is the same sum, but the subtraction of neighbouring values is exact for
// smooth fields, so rounding scales with the differences of x rather than x
// itself: one power of the mesh size better for stiffness-like factors (whose
// rows nearly sum to zero).  Mass-like S factors keep the plain form.
//
// Kernel (one CTA = 128 columns x TA rows of Y, 128 threads, one column per
// thread):
//   1. stage the X tile with its K-halo in shared memory: in the PCG form two
//      TMA loads (Z and the previous direction Q_prev, 16-byte aligned boxes,
//      zero fill outside), then X = Z + beta Q_prev in shared memory and the
//      CTA's own rows/columns of the new direction written back with 16-byte
//      stores; otherwise plain coalesced loads;
//   2. stream down the rows: for each new input row every thread forms the
//      t-pass values W_i[r][b] = (X T_i^T)[r][b] for all terms (the 2K neighbour
//      differences are shared by all terms) and keeps the last 2K+1 rows of
//      each in a register ring (compile-time indices after unrolling by 2K+1);
//   3. s-pass Y[a][b] = sum_i (S_i W_i)[a][b] with the row coefficients read as
//      shared-memory broadcasts.
//   Each X element is read from HBM once plus a K-row/column halo per tile, each
//   Y element is written once.
//   Fused epilogues: Y = Bm - L(X) (FP64 true residual) and an FP64 partial of
//   <X, Y> (or <Y, Y>) per CTA; in the PCG form the last CTA of each instance
//   sums the partials in a fixed order and sets alpha = <R,Z>/<Q,L(Q)>.
#pragma once
#include "internal.h"

#include <type_traits>

namespace mofem_apply_impl {

constexpr int TB = 128;   // columns per CTA (= threads)
constexpr int XPAD = 4;   // aligned left halo of the staged tile (>= K)
constexpr int WCT = TB + 2 * XPAD;   // staged columns in the TMA path
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

template <int K>
struct Geo {
    static constexpr int P = 2 * K + 1;
    static constexpr int MR_G = (64 + P - 1) / P;   // generic path: ~64 rows
    static constexpr int TA_G = MR_G * P;
    static constexpr int MR_T = (36 + P - 1) / P;   // TMA path: ~36-42 rows (two staging buffers)
    static constexpr int TA_T = MR_T * P;
};

// Terms whose S factor is stiffness- or convection-like (difference form in the s-pass).
template <int NT>
struct DiffMask {
    static constexpr unsigned value = NT == 5 ? 0x19u : (NT == 8 ? 0xF1u : 0u);
};

using KArgs = ApplyArgs;

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

// Shared-memory compute of one tile, common to both staging paths.
//   Xs: staged input with row stride ws; this thread's centre column is at
//   c0 + tid, input column b + l - K at c0 + tid + l - K; staged row lr holds
//   input row a0 - K + lr (+ off).
template <typename T, int K, int NT, bool TSMEM, int TA, int MODE>
__device__ __forceinline__ double compute_tile(const T* Xs, int ws, int c0, const T* Ss, const T* Ts,
                                               const T (&tc)[TSMEM ? 1 : NT][TSMEM ? 1 : (2 * K + 1)],
                                               T* Y, const T* Bm, int y_ld, int a0, int b, bool col_ok,
                                               int rows_out, bool want_xy) {
    constexpr int P = 2 * K + 1;
    constexpr int MR = TA / P;
    constexpr unsigned DM = DiffMask<NT>::value;
    constexpr int SR = ((NT * P + 3) / 4) * 4;   // padded S row (16-byte aligned)
    const int tid = threadIdx.x;
    auto tcoef = [&](int i, int l) -> T {
        if constexpr (TSMEM) return Ts[(i * P + l) * TB + tid];
        else return tc[i][l];
    };
    // Term 0, (K_s[h] + gamma M_s[h]) (x) M_t, is the one whose t-factor is a mass
    // and whose s-factor is a stiffness: an FP32 rounding of the t-pass value would
    // be amplified by the s-stiffness by ~(mesh size)^-2 on smooth fields.  With
    // D = diag(rowsum M_t) and N = D^{-1}(M_t - D) (zero row sums), the t-pass is
    // split exactly as X M_t^T = D (X + X N^T): the s-pass is applied separately to
    // the exact staged column X and to the small W' = X N^T, and the sum is scaled
    // by D_b once.  Other terms first apply their stiffness/derivative factor.
    constexpr bool SPLIT0 = NT > 1 && sizeof(T) == 4;   // FP64 keeps enough digits in the t-mass product
    T ring[NT][P];
    T xr0[SPLIT0 ? P : 1];
    T n0[SPLIT0 ? P : 1];   // N coefficients of term 0 (row b of D^{-1} M_t off the diagonal)
    T d0 = (T)1;
    if constexpr (SPLIT0) {
        d0 = tcoef(0, K);
        const T dinv = d0 != (T)0 ? (T)1 / d0 : (T)0;
#pragma unroll
        for (int l = 0; l < P; ++l) n0[l] = (l == K) ? (T)0 : tcoef(0, l) * dinv;
    }
    auto tpass = [&](int lr, int slot) {
        T xv[P];
        const T* row = Xs + lr * ws + c0 + tid - K;
#pragma unroll
        for (int l = 0; l < P; ++l) xv[l] = row[l];
        const T xc = xv[K];
        if constexpr (SPLIT0) xr0[slot] = xc;
#pragma unroll
        for (int l = 0; l < P; ++l)
            if (l != K) xv[l] -= xc;
        if constexpr (SPLIT0) {
            T w = (T)0;
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = fma(n0[l], xv[l], w);
            ring[0][slot] = w;
        }
#pragma unroll
        for (int i = SPLIT0 ? 1 : 0; i < NT; ++i) {
            T w = tcoef(i, K) * xc;
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = fma(tcoef(i, l), xv[l], w);
            ring[i][slot] = w;
        }
    };
#pragma unroll
    for (int lr = 0; lr < 2 * K; ++lr) tpass(lr, lr);
    T accT = (T)0;   // per-thread partial of <X, Y> or <Y, Y> (working precision; few terms)
    for (int m = 0; m < MR; ++m) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int al = m * P + u;
            tpass(al + 2 * K, (u + P - 1) % P);
            const T* srow = Ss + al * SR;
            T y = (T)0;
            if constexpr (SPLIT0) {
                const T xc = xr0[(u + K) % P], wc = ring[0][(u + K) % P];
                T ya = srow[K] * xc, yb = srow[K] * wc;
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (j != K) {
                        ya = fma(srow[j], xr0[(u + j) % P] - xc, ya);
                        yb = fma(srow[j], ring[0][(u + j) % P] - wc, yb);
                    }
                y = d0 * (ya + yb);
            }
#pragma unroll
            for (int i = SPLIT0 ? 1 : 0; i < NT; ++i) {
                const T wc = ring[i][(u + K) % P];
                y = fma(srow[i * P + K], wc, y);
                if ((DM >> i) & 1u) {
#pragma unroll
                    for (int j = 0; j < P; ++j)
                        if (j != K) y = fma(srow[i * P + j], ring[i][(u + j) % P] - wc, y);
                } else {
#pragma unroll
                    for (int j = 0; j < P; ++j)
                        if (j != K) y = fma(srow[i * P + j], ring[i][(u + j) % P], y);
                }
            }
            const int ar = a0 + al;
            if (col_ok && ar < rows_out) {
                const size_t o = (size_t)ar * y_ld + b;
                if (MODE == APPLY_RESIDUAL) {
                    y = Bm[o] - y;
                    accT = fma(y, y, accT);
                } else if (want_xy) {
                    accT = fma(Xs[(al + K) * ws + c0 + tid], y, accT);
                }
                Y[o] = y;
            }
        }
    }
    return (double)accT;
}

template <typename T, int K, int NT, bool TSMEM, int TA>
__device__ __forceinline__ void load_coefs(const T* Stab, const T* Ttab, int q_s, int q_t, int a0, int b0, T* Ss,
                                           T* Ts, T (&tc)[TSMEM ? 1 : NT][TSMEM ? 1 : (2 * K + 1)]) {
    constexpr int P = 2 * K + 1;
    constexpr int SR = ((NT * P + 3) / 4) * 4;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < TA * SR; idx += TB) {
        const int r = idx / SR, e = idx - r * SR;
        const int gr = a0 + r;
        T v = (T)0;
        if (e < NT * P && gr < q_s) v = Stab[(size_t)e * q_s + gr];   // e = i * P + j
        Ss[idx] = v;
    }
    const int b = b0 + tid;
    if constexpr (TSMEM) {
        for (int idx = tid; idx < NT * P * TB; idx += TB) {
            const int il = idx / TB, c = idx - il * TB;
            Ts[idx] = (b0 + c < q_t) ? Ttab[(size_t)il * q_t + b0 + c] : (T)0;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int l = 0; l < P; ++l) tc[i][l] = (b < q_t) ? Ttab[((size_t)i * P + l) * q_t + b] : (T)0;
    }
}

template <int NTH>
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int w = 0; w < NTH / 32; ++w) s += red[w];
    return s;
}

// ---------------------------------------------------------------------------
// Generic path: any leading dimension, plain loads (mofem_apply, the RHS, the
// FP64 true residual).
template <typename T, int K, int NT, int MODE, bool TSMEM>
__global__ void __launch_bounds__(TB) k_apply(KArgs a) {
    constexpr int P = 2 * K + 1, TA = Geo<K>::TA_G, HR = TA + 2 * K, WC = TB + 2 * K;
    constexpr int SR = ((NT * P + 3) / 4) * 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Xs = reinterpret_cast<T*>(smem_raw);   // [HR][WC]
    T* Ss = Xs + ((HR * WC + 3) / 4) * 4;     // [TA][SR]
    T* Ts = Ss + TA * SR;                     // [NT][P][TB] (TSMEM)
    __shared__ double red[TB / 32];
    const int tid = threadIdx.x, inst = blockIdx.z;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * TB;
    const T* X = reinterpret_cast<const T*>(a.X) + (size_t)inst * a.x_bs;
    const int r_base = a0 + a.off - K, c_base = b0 + a.off - K;
    // one warp per staged row at a time: coalesced, no division per element
    for (int r = tid / 32; r < HR; r += TB / 32) {
        const int gr = r_base + r;
        const bool rok = gr >= 0 && gr < a.rows_in;
        for (int cc = tid & 31; cc < WC; cc += 32) {
            const int gc = c_base + cc;
            Xs[r * WC + cc] = (rok && gc >= 0 && gc < a.cols_in) ? X[(size_t)gr * a.x_ld + gc] : (T)0;
        }
    }
    T tc[TSMEM ? 1 : NT][TSMEM ? 1 : P];
    load_coefs<T, K, NT, TSMEM, TA>(reinterpret_cast<const T*>(a.S) + (size_t)inst * a.s_bs,
                                    reinterpret_cast<const T*>(a.T), a.rows_out, a.cols_out, a0, b0, Ss, Ts, tc);
    __syncthreads();
    const int b = b0 + tid;
    double acc = compute_tile<T, K, NT, TSMEM, TA, MODE>(
        Xs, WC, K, Ss, Ts, tc, reinterpret_cast<T*>(a.Y) + (size_t)inst * a.y_bs,
        reinterpret_cast<const T*>(a.Bm) + (size_t)inst * a.y_bs, a.y_ld, a0, b, b < a.cols_out, a.rows_out,
        a.partial != nullptr && a.off == 0);
    if (a.partial) {
        double s = block_sum<TB>(acc, red);
        if (tid == 0) a.partial[(size_t)inst * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// PCG path: internal buffers (16-byte aligned rows), TMA staging, fused
// search-direction update Q = Z + beta Q_prev, partial <Q, L(Q)> and the
// last-CTA finalisation alpha = <R, Z> / <Q, L(Q)>.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(a, parity))
        if (gtimer() - t0 > WAIT_LIMIT_NS) return false;
    return true;
}

template <typename T, int K, int NT, bool TSMEM>
__global__ void __launch_bounds__(TB) k_apply_pcg(const __grid_constant__ CUtensorMap mZ,
                                                  const __grid_constant__ CUtensorMap mQ, ApplyPcgArgs a) {
    constexpr int P = 2 * K + 1, TA = Geo<K>::TA_T, HR = TA + 2 * K;
    constexpr int BUF = HR * WCT;   // elements per staging buffer
    constexpr int BUFP = ((BUF * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);   // 128-byte multiple
    constexpr int SR = ((NT * P + 3) / 4) * 4;
    // TMA destinations must be 128-byte aligned: align the dynamic region by hand
    // (static shared variables may precede it) and round each buffer up to 128 B.
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem_base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    T* Zs = reinterpret_cast<T*>(smem_base);  // [HR][WCT]  -> becomes X = Z + beta Q
    T* Qs = Zs + BUFP;                        // [HR][WCT]
    T* Ss = Qs + BUFP;                        // [TA][SR]
    T* Ts = Ss + TA * SR;                     // [NT][P][TB] (TSMEM)
    __shared__ __align__(8) unsigned long long bar;
    __shared__ double red[TB / 32];
    __shared__ T beta_s;
    __shared__ int fail_s;
    __shared__ int last_s;
    const int tid = threadIdx.x, inst = blockIdx.z;
    PcgScalars* sc = a.sc + inst;
    if (a.use_sc && !sc->active) return;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * TB;
    const uint32_t bar_a = smem_u32(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        beta_s = (a.use_sc && sc->iters > 0) ? (T)sc->beta : (T)0;
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t bytes = 2u * BUF * sizeof(T);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(bytes) : "memory");
        const int x0 = b0 - XPAD, y0 = a0 - K;
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Zs)), "l"(reinterpret_cast<uint64_t>(&mZ)), "r"(bar_a), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Qs)), "l"(reinterpret_cast<uint64_t>(&mQ)), "r"(bar_a), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
    }
    T tc[TSMEM ? 1 : NT][TSMEM ? 1 : P];
    load_coefs<T, K, NT, TSMEM, TA>(reinterpret_cast<const T*>(a.S) + (size_t)inst * a.s_bs,
                                    reinterpret_cast<const T*>(a.T), a.q, a.q, a0, b0, Ss, Ts, tc);
    if (!mbar_wait_bounded(bar_a, 0)) atomicOr(&fail_s, 1);
    __syncthreads();
    if (fail_s) {   // the copies never completed: record it and leave without touching them
        if (tid == 0) atomicOr(a.status, DEV_ERR_TIMEOUT);
        return;
    }
    // X = Z + beta Q_prev over the staged tile; write the owned block of the new direction
    {
        const T beta = beta_s;
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int VW = 16 / sizeof(T);
        V* zv = reinterpret_cast<V*>(Zs);
        const V* qv = reinterpret_cast<const V*>(Qs);
        for (int i = tid; i < BUF / VW; i += TB) {
            V z = zv[i];
            const V qq = qv[i];
            if constexpr (VW == 4) {
                z.x += beta * qq.x; z.y += beta * qq.y; z.z += beta * qq.z; z.w += beta * qq.w;
            } else {
                z.x += beta * qq.x; z.y += beta * qq.y;
            }
            zv[i] = z;
        }
        __syncthreads();
        T* Qn = reinterpret_cast<T*>(a.Qnew) + (size_t)inst * a.bs;
        constexpr int VPR = TB / VW;   // vectors per owned row
        const int rows_own = min(TA, a.q - a0);
        const int cols_lim = min(TB, a.ld - b0);   // stay inside the padded row
        for (int i = tid; i < rows_own * VPR; i += TB) {
            const int r = i / VPR, cv = (i - r * VPR) * VW;
            if (cv < cols_lim)
                *reinterpret_cast<V*>(Qn + (size_t)(a0 + r) * a.ld + b0 + cv) =
                    *reinterpret_cast<const V*>(Zs + (r + K) * WCT + XPAD + cv);
        }
    }
    const int b = b0 + tid;
    double acc = compute_tile<T, K, NT, TSMEM, TA, APPLY_PLAIN>(
        Zs, WCT, XPAD, Ss, Ts, tc, reinterpret_cast<T*>(a.LQ) + (size_t)inst * a.bs, nullptr, a.ld, a0, b, b < a.q,
        a.q, true);
    double s = block_sum<TB>(acc, red);
    // partial, then the last CTA of this instance finalises alpha (fixed-order sum)
    const int nblk = gridDim.x * gridDim.y;
    if (tid == 0) {
        a.partial[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(a.counter + inst, 1u);
        last_s = (t == (unsigned)nblk - 1) ? 1 : 0;
    }
    __syncthreads();
    if (last_s && tid < 32) {
        __threadfence();
        const double qlq = warp_sum_partials(a.partial + (size_t)inst * nblk, nblk);
        if (tid == 0) {
            a.counter[inst] = 0;
            double al = sc->rz / qlq;
            if (!(qlq > 0.0) || !isfinite(al)) {
                if (a.use_sc) {
                    sc->status |= isfinite(qlq) ? DEV_ERR_BREAKDOWN : DEV_ERR_NONFINITE;
                    sc->active = 0;
                }
                al = 0.0;
            }
            sc->alpha = al;
        }
    }
}

template <typename T, int K, int NT, bool TSMEM>
size_t smem_generic() {
    constexpr int P = 2 * K + 1, TA = Geo<K>::TA_G, HR = TA + 2 * K, WC = TB + 2 * K;
    constexpr int SR = ((NT * P + 3) / 4) * 4;
    size_t n = (size_t)((HR * WC + 3) / 4) * 4 + (size_t)TA * SR + (TSMEM ? (size_t)NT * P * TB : 0);
    return n * sizeof(T);
}

template <typename T, int K, int NT, bool TSMEM>
size_t smem_pcg() {
    constexpr int P = 2 * K + 1, TA = Geo<K>::TA_T, HR = TA + 2 * K;
    constexpr int SR = ((NT * P + 3) / 4) * 4;
    constexpr int BUFP = ((HR * WCT * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
    size_t n = 2 * (size_t)BUFP + (size_t)TA * SR + (TSMEM ? (size_t)NT * P * TB : 0);
    return n * sizeof(T) + 128;   // + alignment slack of the dynamic base
}

template <typename T, int K, int NT, int MODE, bool TSMEM>
mofem_status launch_t(const KArgs& a, int batch, cudaStream_t st) {
    const size_t sm = smem_generic<T, K, NT, TSMEM>();
    auto kern = k_apply<T, K, NT, MODE, TSMEM>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];   // per instantiation and device
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)sm, attr_done));
    dim3 grid((a.cols_out + TB - 1) / TB, (a.rows_out + Geo<K>::TA_G - 1) / Geo<K>::TA_G, batch);
    kern<<<grid, TB, sm, st>>>(a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

template <typename T, int K, int NT, bool TSMEM>
mofem_status launch_pcg_t(const CUtensorMap& mZ, const CUtensorMap& mQ, const ApplyPcgArgs& a, int batch,
                          cudaStream_t st) {
    const size_t sm = smem_pcg<T, K, NT, TSMEM>();
    auto kern = k_apply_pcg<T, K, NT, TSMEM>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)sm, attr_done));
    dim3 grid((a.q + TB - 1) / TB, (a.q + Geo<K>::TA_T - 1) / Geo<K>::TA_T, batch);
    kern<<<grid, TB, sm, st>>>(mZ, mQ, a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
