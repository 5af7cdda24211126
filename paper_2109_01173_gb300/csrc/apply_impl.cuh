// Banded multiterm operator apply  Y = sum_i S_i X T_i^T  (Sec. 5, operator L~;
// Eq. laplace_cap-shaped-domain_sylvester), the hot operator of every MO-PCG
// iteration.
//
// Data: X, Y row-major (rows = s-nodes a, columns = t-nodes b).  S_i and T_i are
// banded with half-bandwidth K (the element degree), stored diagonal-major:
// tab[i][j][r] = M_i[r][r + off + j - K], j = 0..2K.  Out-of-range entries are 0.
//
// Kernel design (one CTA = 128 columns x TA rows of Y, 128 threads, one column
// per thread):
//   1. stage the X tile with its K-halo in shared memory (zero outside X);
//      optional fused prologue X = Z + beta * Q_prev that also writes the new
//      search direction (the PCG direction update);
//   2. stream down the rows; for each new input row r every thread forms the
//      t-pass values W_i[r][b] = sum_l T_i[b][l] X[r][b + l - K] for all terms and
//      keeps the last 2K+1 of them in a register ring (indices are compile-time
//      after unrolling by 2K+1 rows);
//   3. the s-pass Y[a][b] = sum_i sum_j S_i[a][j] W_i[a + j - K][b] reads the
//      row coefficients S_i[a][*] as shared-memory broadcasts.
//   Each X element is read from HBM once (plus a K-row halo per tile) and each Y
//   element written once: the algorithmic traffic of the apply.
//   Optional fused epilogues: Y = Bm - L(X) (true residual) and an FP64 partial
//   of <X, Y> or <Y, Y> per CTA (deterministic fixed-order reduction later).
#pragma once
#include "internal.h"

namespace mofem_apply_impl {

constexpr int TB = 128;   // columns per CTA (= threads)

template <int K>
struct Geo {
    static constexpr int P = 2 * K + 1;
    static constexpr int MR = (64 + P - 1) / P;   // ring periods per CTA
    static constexpr int TA = MR * P;             // output rows per CTA
    static constexpr int HR = TA + 2 * K;         // staged input rows
    static constexpr int WC = TB + 2 * K;         // staged input columns
};

using KArgs = ApplyArgs;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order sum of n partials by one warp (all lanes return the total).
__device__ __forceinline__ double warp_sum_partials(const double* p, int n) {
    double s = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) s += p[i];
    return warp_sum(s);
}

template <typename T, int K, int NT, int MODE, bool TSMEM>
__global__ void __launch_bounds__(TB) k_apply(KArgs a) {
    using G = Geo<K>;
    constexpr int P = G::P, TA = G::TA, HR = G::HR, WC = G::WC, MR = G::MR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Xs = reinterpret_cast<T*>(smem_raw);                 // [HR][WC]
    T* Ss = Xs + HR * WC;                                   // [TA][NT][P]
    T* Ts = Ss + TA * NT * P;                               // [NT][P][TB] (TSMEM)
    __shared__ double red[TB / 32];
    __shared__ T beta_s;

    const int tid = threadIdx.x;
    const int inst = blockIdx.z;
    const int a0 = blockIdx.y * TA;
    const int b0 = blockIdx.x * TB;
    const int q_t = a.cols_out;     // rows of the T tables
    const int q_s = a.rows_out;     // rows of the S tables

    if (MODE == APPLY_QUPDATE) {
        if (a.sc && !a.sc[inst].active) return;
        if (tid < 32) {
            double beta = 0.0;
            if (a.sc[inst].iters > 0) {
                double rzc = warp_sum_partials(a.rz_cur + (size_t)inst * a.n_rz, a.n_rz);
                double rzp = warp_sum_partials(a.rz_prev + (size_t)inst * a.n_rz, a.n_rz);
                double rzo = a.flex ? warp_sum_partials(a.rzo + (size_t)inst * a.n_rzo, a.n_rzo) : 0.0;
                beta = (rzc - rzo) / rzp;
                if (!(fabs(beta) < 1e300)) beta = 0.0;   // guarded; the control kernel flags non-finite
            }
            if (tid == 0) beta_s = (T)beta;
        }
        __syncthreads();
    }

    const T* X = reinterpret_cast<const T*>(a.X) + (size_t)inst * a.x_bs;
    const T* Zp = reinterpret_cast<const T*>(a.Z) + (size_t)inst * a.x_bs;
    T* Xn = reinterpret_cast<T*>(a.Xnew) + (size_t)inst * a.x_bs;
    const T* Stab = reinterpret_cast<const T*>(a.S) + (size_t)inst * a.s_bs;
    const T* Ttab = reinterpret_cast<const T*>(a.T);

    // ---- stage X tile (rows a0+off-K .., cols b0+off-K ..) ----
    const int r_base = a0 + a.off - K, c_base = b0 + a.off - K;
    for (int idx = tid; idx < HR * WC; idx += TB) {
        int r = idx / WC, cc = idx - r * WC;
        int gr = r_base + r, gc = c_base + cc;
        T v = (T)0;
        if (gr >= 0 && gr < a.rows_in && gc >= 0 && gc < a.cols_in) {
            size_t o = (size_t)gr * a.x_ld + gc;
            if (MODE == APPLY_QUPDATE) {
                v = Zp[o] + beta_s * X[o];
                // the CTA owns rows [a0, a0+TA) and columns [b0, b0+TB) of the new direction
                if (gr >= a0 && gr < a0 + TA && gc >= b0 && gc < b0 + TB) Xn[o] = v;
            } else {
                v = X[o];
            }
        }
        Xs[idx] = v;
    }
    // ---- S coefficients of the tile rows ----
    for (int idx = tid; idx < TA * NT * P; idx += TB) {
        int r = idx / (NT * P), rem = idx - r * NT * P;
        int i = rem / P, j = rem - i * P;
        int gr = a0 + r;
        Ss[idx] = (gr < q_s) ? Stab[((size_t)i * P + j) * q_s + gr] : (T)0;
    }
    const int b = b0 + tid;
    T tc[TSMEM ? 1 : NT][TSMEM ? 1 : P];
    if (TSMEM) {
        for (int idx = tid; idx < NT * P * TB; idx += TB) {
            int il = idx / TB, c = idx - il * TB;
            Ts[idx] = (b0 + c < q_t) ? Ttab[(size_t)il * q_t + b0 + c] : (T)0;
        }
    } else {
#pragma unroll
        for (int i = 0; i < (TSMEM ? 1 : NT); ++i)
#pragma unroll
            for (int l = 0; l < (TSMEM ? 1 : P); ++l)
                tc[i][l] = (b < q_t) ? Ttab[((size_t)i * P + l) * q_t + b] : (T)0;
    }
    __syncthreads();

    auto tcoef = [&](int i, int l) -> T {
        if (TSMEM) return Ts[(i * P + l) * TB + tid];
        return tc[TSMEM ? 0 : i][TSMEM ? 0 : l];
    };

    T ring[NT][P];
    auto tpass = [&](int lr, int slot) {
        T xv[P];
#pragma unroll
        for (int l = 0; l < P; ++l) xv[l] = Xs[lr * WC + tid + l];
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            T w = (T)0;
#pragma unroll
            for (int l = 0; l < P; ++l) w = fma(tcoef(i, l), xv[l], w);
            ring[i][slot] = w;
        }
    };

#pragma unroll
    for (int lr = 0; lr < 2 * K; ++lr) tpass(lr, lr);

    T* Y = reinterpret_cast<T*>(a.Y) + (size_t)inst * a.y_bs;
    const T* Bm = reinterpret_cast<const T*>(a.Bm) + (size_t)inst * a.y_bs;
    const bool col_ok = b < a.cols_out;
    double acc = 0.0;

    for (int m = 0; m < MR; ++m) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int al = m * P + u;
            tpass(al + 2 * K, (u + P - 1) % P);
            const T* srow = Ss + al * NT * P;
            T y = (T)0;
#pragma unroll
            for (int i = 0; i < NT; ++i)
#pragma unroll
                for (int j = 0; j < P; ++j) y = fma(srow[i * P + j], ring[i][(u + j) % P], y);
            const int ar = a0 + al;
            if (col_ok && ar < a.rows_out) {
                size_t o = (size_t)ar * a.y_ld + b;
                if (MODE == APPLY_RESIDUAL) {
                    y = Bm[o] - y;
                    acc += (double)y * (double)y;
                } else if (a.partial) {
                    // <X, Y>: X[ar][b] is the staged value at row ar-(a0+off-K), column tid+K
                    acc += (double)Xs[(al + K) * WC + tid + K] * (double)y;
                }
                Y[o] = y;
            }
        }
    }

    if (a.partial) {
        acc = warp_sum(acc);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < TB / 32; ++w) s += red[w];
            const int nblk = gridDim.x * gridDim.y;
            a.partial[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}

template <typename T, int K, int NT, bool TSMEM>
size_t smem_bytes() {
    using G = Geo<K>;
    size_t n = (size_t)G::HR * G::WC + (size_t)G::TA * NT * G::P + (TSMEM ? (size_t)NT * G::P * TB : 0);
    return n * sizeof(T);
}

template <typename T, int K, int NT, int MODE, bool TSMEM>
mofem_status launch_t(const KArgs& a, int batch, cudaStream_t st) {
    using G = Geo<K>;
    size_t sm = smem_bytes<T, K, NT, TSMEM>();
    auto kern = k_apply<T, K, NT, MODE, TSMEM>;
    static bool attr_done = false;   // per instantiation
    if (!attr_done) {
        MOFEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr_done = true;
    }
    dim3 grid((a.cols_out + TB - 1) / TB, (a.rows_out + G::TA - 1) / G::TA, batch);
    kern<<<grid, TB, sm, st>>>(a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
