// Residual update of the mixed refinement in double-float arithmetic:
//
//     R64 <- R64 - L(d),   L(d) = sum_i S_i d T_i^T   (Sec. 5, operator L~)
//
// for the correction d = hi + lo + alpha_pend Q_pend - err of one refinement step
// (the inner solve's double-float accumulator, its pending last term, and the exact
// rounding error err of the FP64 iterate's update U <- fl(U + d), so that R tracks
// B - L(U) of the stored iterate).  From the second refinement step on this
// replaces the FP64 recomputation R = B - L(U): |d| is ~1e-5 |U| there, so an
// evaluation of L(d) with ~2^-46 relative arithmetic (double-float: exact FMA
// products, TwoSum accumulation) is accurate to ~1e-13 of ||B||, and it runs on
// the FP32 pipes (FP64 throughput on this GPU is a small fraction of FP32).  Plain (not
// difference) form: the coefficient tables are the plain banded factors split
// into FP32 (hi, lo) pairs at setup.
//
// Kernel: one CTA = 128 columns x TA rows, one column per thread; the correction
// tile (with its K-halo) is formed in shared memory as (hi, lo) pairs, the t-pass
// values of all terms for each new row enter a register ring of the last 2K+1
// rows, the s-pass reads the row's coefficients as shared-memory broadcasts.
// Output: R64 updated in place and one FP64 partial of ||R64||^2 per CTA.
#include "internal.h"

namespace {

constexpr int DTB = 128;

template <int K>
struct DGeo {
    static constexpr int P = 2 * K + 1;
    static constexpr int MR = (32 + P - 1) / P;
    static constexpr int TA = MR * P;
    static constexpr int HR = TA + 2 * K;
    static constexpr int WC = DTB + 2 * K;
};

struct DfArgs {
    const float* hi; const float* lo; const float* qp;   // correction parts, [batch][q][ld]
    const float* err;                                    // rounding error of the fold (or null)
    const PcgScalars* sc;                                // alpha_pend per instance
    const float* Sh; const float* Sl; long long s_bs;    // S tables, hi / lo planes, [batch][NT][P][q]
    const float* Th; const float* Tl;                    // T tables, hi / lo planes, [NT][P][q]
    double* R; long long bs; int ld, q;
    double* partial;
};

struct dfl {
    float h, l;
};

// s += (ah + al)(bh + bl): high product exact by FMA, cross terms in FP32,
// TwoSum of the high parts, renormalised.
__device__ __forceinline__ void acc_prod(dfl& s, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = s.h + p;
    const float v = t - s.h;
    e += (s.h - (t - v)) + (p - v);
    e += s.l;
    s.h = t + e;
    s.l = e - (s.h - t);
}

template <int K, int NT>
__global__ void __launch_bounds__(DTB) k_resid_df(DfArgs a) {
    using G = DGeo<K>;
    constexpr int P = G::P, TA = G::TA, MR = G::MR, HR = G::HR, WC = G::WC, NTP = NT * P;
    extern __shared__ __align__(16) float dsm[];
    float* xh = dsm;                     // [HR][WC]
    float* xl = xh + HR * WC;            // [HR][WC]
    float* s_h = xl + HR * WC;           // [TA][NTP]
    float* s_l = s_h + TA * NTP;         // [TA][NTP]
    __shared__ double red[DTB / 32];
    const int tid = threadIdx.x, inst = blockIdx.z;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * DTB;
    const int q = a.q;
    const double apd = a.sc ? a.sc[inst].alpha_pend : 0.0;
    const float aph = (float)apd, apl = (float)(apd - (double)aph);   // alpha_pend as a double-float
    const float* hi = a.hi + (size_t)inst * a.bs;
    const float* lo = a.lo + (size_t)inst * a.bs;
    const float* qp = a.qp + (size_t)inst * a.bs;
    const float* er = a.err ? a.err + (size_t)inst * a.bs : nullptr;
    // correction tile with halo: d = (hi, lo) + ap * qp - err (exact products, TwoSum), zero outside
    for (int r = tid / 32; r < HR; r += DTB / 32) {
        const int gr = a0 - K + r;
        const bool rok = gr >= 0 && gr < q;
        for (int cc = tid & 31; cc < WC; cc += 32) {
            const int gc = b0 - K + cc;
            dfl x{0.f, 0.f};
            if (rok && gc >= 0 && gc < q) {
                const size_t o = (size_t)gr * a.ld + gc;
                x.h = hi[o];
                x.l = lo[o];
                if (aph != 0.f) acc_prod(x, aph, apl, qp[o], 0.f);
                if (er) acc_prod(x, er[o], 0.f, -1.f, 0.f);
            }
            xh[r * WC + cc] = x.h;
            xl[r * WC + cc] = x.l;
        }
    }
    for (int idx = tid; idx < TA * NTP; idx += DTB) {
        const int r = idx / NTP, e = idx - r * NTP;
        const int gr = a0 + r;
        float vh = 0.f, vl = 0.f;
        if (gr < q) {
            const size_t o = (size_t)inst * a.s_bs + (size_t)e * q + gr;
            vh = a.Sh[o];
            vl = a.Sl[o];
        }
        s_h[idx] = vh;
        s_l[idx] = vl;
    }
    const int b = b0 + tid;
    float th[NT][P], tl[NT][P];
#pragma unroll
    for (int i = 0; i < NT; ++i)
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const size_t o = (size_t)(i * P + l) * q + b;
            th[i][l] = b < q ? a.Th[o] : 0.f;
            tl[i][l] = b < q ? a.Tl[o] : 0.f;
        }
    __syncthreads();
    dfl ring[NT][P];
    auto tpass = [&](int lr, int slot) {
        const float* rh = xh + lr * WC + tid;   // staged column of input b + l - K is tid + l
        const float* rl = xl + lr * WC + tid;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            dfl w{0.f, 0.f};
#pragma unroll
            for (int l = 0; l < P; ++l) acc_prod(w, th[i][l], tl[i][l], rh[l], rl[l]);
            ring[i][slot] = w;
        }
    };
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) tpass(r, r);
    float rs = 0.f;
    double* Rg = a.R + (size_t)inst * a.bs;
#pragma unroll 1
    for (int m = 0; m < MR; ++m) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int al = m * P + u;
            tpass(al + 2 * K, (u + P - 1) % P);
            const float* ch = s_h + al * NTP;
            const float* cl = s_l + al * NTP;
            // one accumulation chain per term (independent chains hide the FP32 latency)
            dfl ys[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) ys[i] = dfl{0.f, 0.f};
#pragma unroll
            for (int j = 0; j < P; ++j)
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const dfl& w = ring[i][(u + j) % P];
                    acc_prod(ys[i], ch[i * P + j], cl[i * P + j], w.h, w.l);
                }
            dfl y = ys[0];
#pragma unroll
            for (int i = 1; i < NT; ++i) acc_prod(y, ys[i].h, ys[i].l, 1.f, 0.f);
            const int gr = a0 + al;
            if (gr < q && b < q) {
                const size_t o = (size_t)gr * a.ld + b;
                const double r = Rg[o] - ((double)y.h + (double)y.l);
                Rg[o] = r;
                const float rf = (float)r;
                rs = fmaf(rf, rf, rs);
            }
        }
    }
    double v = (double)rs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < DTB / 32; ++w) t += red[w];
        a.partial[(size_t)inst * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

template <int K>
constexpr int df_rows() { return DGeo<K>::TA; }

template <int K, int NT>
mofem_status launch_df_t(const DfArgs& a, int batch, int* nblk, cudaStream_t st) {
    using G = DGeo<K>;
    const size_t smem = sizeof(float) * (2 * (size_t)G::HR * G::WC + 2 * (size_t)G::TA * NT * G::P);
    static bool attr = false;
    if (!attr) {
        MOFEM_CUDA_TRY(cudaFuncSetAttribute(k_resid_df<K, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    dim3 grid((a.q + DTB - 1) / DTB, (a.q + G::TA - 1) / G::TA, batch);
    *nblk = grid.x * grid.y;
    k_resid_df<K, NT><<<grid, DTB, smem, st>>>(a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

template <int K>
mofem_status df_nt(int nt, const DfArgs& a, int batch, int* nblk, cudaStream_t st) {
    if (nt == 5) return launch_df_t<K, 5>(a, batch, nblk, st);
    if constexpr (8 * (2 * K + 1) <= 40)
        if (nt == 8) return launch_df_t<K, 8>(a, batch, nblk, st);
    return MOFEM_ERR_UNSUPPORTED;
}

}  // namespace

int residual_update_df_ctas(int K, int q) {
    if (K < 1 || K > 3) return 0;
    const int ta = K == 1 ? df_rows<1>() : K == 2 ? df_rows<2>() : df_rows<3>();
    return ((q + DTB - 1) / DTB) * ((q + ta - 1) / ta);
}

// Forms served: the ring and the T coefficients in registers (NT * (2K+1) <= 40,
// as the packed FP32 apply); others return MOFEM_ERR_UNSUPPORTED and the caller
// recomputes the residual in FP64.
mofem_status launch_residual_update_df(const mofem_ctx* c, const float* hi, const float* lo, const float* Qpend,
                                       const float* err, double* R, double* partial, int* nblk, cudaStream_t st) {
    if (c->NT * (2 * c->K + 1) > 40 || !c->Sdf || !c->Tdf) return MOFEM_ERR_UNSUPPORTED;
    DfArgs a{};
    a.hi = hi; a.lo = lo; a.qp = Qpend; a.err = err;
    a.sc = c->d_sc;
    const long long sp = (long long)c->batch * c->NT * c->P * c->q;   // S plane size
    const long long tp = (long long)c->NT * c->P * c->q;              // T plane size
    a.Sh = c->Sdf; a.Sl = c->Sdf + sp; a.s_bs = (long long)c->NT * c->P * c->q;
    a.Th = c->Tdf; a.Tl = c->Tdf + tp;
    a.R = R; a.bs = (long long)c->q * c->ld; a.ld = c->ld; a.q = c->q;
    a.partial = partial;
    switch (c->K) {
        case 1: return df_nt<1>(c->NT, a, c->batch, nblk, st);
        case 2: return df_nt<2>(c->NT, a, c->batch, nblk, st);
        case 3: return df_nt<3>(c->NT, a, c->batch, nblk, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}
