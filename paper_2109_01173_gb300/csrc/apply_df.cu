// Residual update of the mixed refinement in double-float arithmetic:
//
//     R64 <- R64 - L(d),   L(d) = sum_i S_i d T_i^T   (Sec. 5, operator L~)
//
// for the step d of one refinement step, given as a double-float pair (dh, dl):
// the FP64 iterate's actual change fl(U + d') - U, which the fold of the inner
// solve's correction d' leaves in the correction buffers, so that R tracks
// B - L(U) of the stored iterate, in place of an FP64 recomputation R = B - L(U)
// (FP64 throughput on this GPU is a small fraction of FP32).  Two kernels:
//   k_resid_df   plain form, for steps after the first: |d| is ~1e-5 |U| there, so
//                an evaluation of L(d) with ~2^-44 relative arithmetic is accurate to
//                ~1e-13 of ||B||; tables: the plain banded factors split into FP32
//                (hi, lo) pairs at setup;
//   k_resid_dfd  difference form, for the step from zero (d of the size of U; see
//                its own comment).
//
// Arithmetic: each product (ah + al)(bh + bl) as ah*bh exactly (FMA residual) plus
// the two cross terms; sums of a chain (2K+1 products, or the NT term results)
// keep the running high part and collect every rounding error, exact by TwoSum,
// in the low part, renormalised once at the end of the chain (error of the chain
// ~ n^2 u^2 max|partial sum|, u = 2^-24).
//
// Kernel: one CTA = 128 columns x TA rows, one column per thread; the step's tile
// (with its K-halo) is staged in shared memory as (hi, lo) pairs, the t-pass
// values of all terms for each new row enter a register ring of the last 2K+1
// rows (shifted by one per row), the s-pass reads the row's coefficients as
// shared-memory broadcasts.
// Output: R64 updated in place and one FP64 partial of ||R64||^2 per CTA.
//
// The same kernel in its second mode evaluates the right-hand side B = M_s F M_t^T
// (Sec. 5, operator R~; one mass term, FP64 nodal F with an index offset from the
// trimmed rows to the node rows) from FP64 input split to double-float on load: the
// mass products have no cancellation, so B comes out to ~2^-46 of each entry
// without the FP64 pipe.
#include "internal.h"

namespace {

constexpr int DTB = 128;

template <int K>
struct DGeo {
    static constexpr int P = 2 * K + 1;
    static constexpr int TA = 32;
    static constexpr int HR = TA + 2 * K;
    static constexpr int WC = DTB + 2 * K;
};

enum { DF_RESID = 0, DF_APPLY64 = 1 };

struct DfArgs {
    const float* dh; const float* dl;                    // the step, [batch][q][ld] (DF_RESID)
    const double* X; long long x_bs; int x_ld;           // FP64 input (DF_APPLY64)
    int rows_in, cols_in, off;                           // input extent; input index = output index + off
    double* Y; long long y_bs; int y_ld;                 // output (DF_APPLY64)
    const float* Sh; const float* Sl; long long s_bs;    // S tables, hi / lo planes, [batch][NT][P][q]
    const float* Th; const float* Tl;                    // T tables, hi / lo planes, [NT][P][q]
    double* R; long long bs; int ld, q;
    double* partial;
};

struct dfl {
    float h, l;
};

// s += (ah + al)(bh + bl); s.l collects the rounding errors (not renormalised).
__device__ __forceinline__ void acc_prod(dfl& s, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = s.h + p;
    const float v = t - s.h;
    const float r = (s.h - (t - v)) + (p - v);   // TwoSum: s.h + p = t + r exactly
    s.h = t;
    s.l += r + e;
}

// (ah + al)(bh + bl) as a new chain: high product and its collected error
__device__ __forceinline__ dfl first_prod(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    return dfl{p, e};
}

// s += x for a double-float x (its low part joins the error collection)
__device__ __forceinline__ void acc_df(dfl& s, dfl x) {
    const float t = s.h + x.h;
    const float v = t - s.h;
    const float r = (s.h - (t - v)) + (x.h - v);
    s.h = t;
    s.l += r + x.l;
}

__device__ __forceinline__ dfl renorm(dfl s) {
    const float h = s.h + s.l;
    return dfl{h, s.l - (h - s.h)};
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& r) {
    s = a + b;
    const float v = s - a;
    r = (a - (s - v)) + (b - v);
}

// x - c for double-float x and c: exact (both high and both low parts by TwoSum),
// then rounded once to double-float.  For differences of neighbouring values of an
// exact input, whose rounding a stiffness factor would amplify by ~(mesh size)^-2.
__device__ __forceinline__ dfl sub_exact(dfl x, dfl c) {
    float s1, r1, s2, r2, t, e1;
    two_sum(x.h, -c.h, s1, r1);
    two_sum(x.l, -c.l, s2, r2);
    two_sum(s1, s2, t, e1);
    const float lo = (e1 + r1) + r2;
    const float h = t + lo;
    return dfl{h, lo - (h - t)};
}

// x - c with the high parts' difference exact and the low parts' rounded once: for
// values that already carry a rounding of that size (t-pass results)
__device__ __forceinline__ dfl sub_df(dfl x, dfl c) {
    float s, r;
    two_sum(x.h, -c.h, s, r);
    const float lo = (x.l - c.l) + r;
    dfl o;
    two_sum(s, lo, o.h, o.l);
    return o;
}

template <int K, int NT, int MODE>
__global__ void __launch_bounds__(DTB, NT * (2 * K + 1) <= 25 ? 4 : 3) k_resid_df(DfArgs a) {
    using G = DGeo<K>;
    constexpr int P = G::P, TA = G::TA, HR = G::HR, WC = G::WC, NTP = NT * P;
    extern __shared__ __align__(16) float dsm[];
    float* xh = dsm;                     // [HR][WC]
    float* xl = xh + HR * WC;            // [HR][WC]
    float* s_h = xl + HR * WC;           // [TA][NTP]
    float* s_l = s_h + TA * NTP;         // [TA][NTP]
    __shared__ double red[DTB / 32];
    const int tid = threadIdx.x, inst = blockIdx.z;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * DTB;
    const int q = a.q;
    // input tile with halo (double-float), zero outside the input
    if constexpr (MODE == DF_RESID) {
        const float* dh = a.dh + (size_t)inst * a.bs;
        const float* dl = a.dl + (size_t)inst * a.bs;
        for (int r = tid / 32; r < HR; r += DTB / 32) {
            const int gr = a0 - K + r;
            const bool rok = gr >= 0 && gr < q;
            for (int cc = tid & 31; cc < WC; cc += 32) {
                const int gc = b0 - K + cc;
                float vh = 0.f, vl = 0.f;
                if (rok && gc >= 0 && gc < q) {
                    const size_t o = (size_t)gr * a.ld + gc;
                    vh = dh[o];
                    vl = dl[o];
                }
                xh[r * WC + cc] = vh;
                xl[r * WC + cc] = vl;
            }
        }
    } else {
        const double* X = a.X + (size_t)inst * a.x_bs;
        for (int r = tid / 32; r < HR; r += DTB / 32) {
            const int gr = a0 - K + r + a.off;
            const bool rok = gr >= 0 && gr < a.rows_in;
            for (int cc = tid & 31; cc < WC; cc += 32) {
                const int gc = b0 - K + cc + a.off;
                float vh = 0.f, vl = 0.f;
                if (rok && gc >= 0 && gc < a.cols_in) {
                    const double x = X[(size_t)gr * a.x_ld + gc];
                    vh = (float)x;
                    vl = (float)(x - (double)vh);
                }
                xh[r * WC + cc] = vh;
                xl[r * WC + cc] = vl;
            }
        }
    }
    for (int idx = tid; idx < TA * NTP; idx += DTB) {   // consecutive rows per thread group: coalesced
        const int e = idx / TA, r = idx - e * TA;
        const int gr = a0 + r;
        float vh = 0.f, vl = 0.f;
        if (gr < q) {
            const size_t o = (size_t)inst * a.s_bs + (size_t)e * q + gr;
            vh = a.Sh[o];
            vl = a.Sl[o];
        }
        s_h[r * NTP + e] = vh;
        s_l[r * NTP + e] = vl;
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
    // ring[i][j] = t-pass value of term i for input row al + j of the current output row al
    // (a register shift per row keeps the loop body one row long: small code)
    dfl ring[NT][P];
    auto tpass = [&](int lr, int slot) {
        const float* rh = xh + lr * WC + tid;   // staged column of input b + l - K is tid + l
        const float* rl = xl + lr * WC + tid;
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            dfl w = first_prod(th[i][0], tl[i][0], rh[0], rl[0]);
#pragma unroll
            for (int l = 1; l < P; ++l) acc_prod(w, th[i][l], tl[i][l], rh[l], rl[l]);
            ring[i][slot] = renorm(w);
        }
    };
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) tpass(r, r + 1);
    float rs = 0.f;
    double* Rg = MODE == DF_RESID ? a.R + (size_t)inst * a.bs : a.Y + (size_t)inst * a.y_bs;
    const int rld = MODE == DF_RESID ? a.ld : a.y_ld;
#pragma unroll 1
    for (int al = 0; al < TA; ++al) {
        // the row's old R is loaded before the row's arithmetic (latency hidden behind it)
        const int gr = a0 + al;
        const bool out = gr < q && b < q;
        const size_t o = (size_t)gr * rld + b;
        const double rold = (MODE == DF_RESID && out) ? Rg[o] : 0.0;
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int j = 0; j + 1 < P; ++j) ring[i][j] = ring[i][j + 1];
        tpass(al + 2 * K, P - 1);
        const float* ch = s_h + al * NTP;
        const float* cl = s_l + al * NTP;
        // one accumulation chain per term (independent chains hide the FP32 latency)
        dfl ys[NT];
#pragma unroll
        for (int i = 0; i < NT; ++i) ys[i] = first_prod(ch[i * P], cl[i * P], ring[i][0].h, ring[i][0].l);
#pragma unroll
        for (int j = 1; j < P; ++j)
#pragma unroll
            for (int i = 0; i < NT; ++i) acc_prod(ys[i], ch[i * P + j], cl[i * P + j], ring[i][j].h, ring[i][j].l);
        dfl y = ys[0];
#pragma unroll
        for (int i = 1; i < NT; ++i) acc_df(y, ys[i]);
        if (out) {
            if constexpr (MODE == DF_RESID) {
                const double r = rold - ((double)y.h + (double)y.l);
                Rg[o] = r;
                const float rf = (float)r;
                rs = fmaf(rf, rf, rs);
            } else {
                Rg[o] = (double)y.h + (double)y.l;
            }
        }
    }
    if constexpr (MODE != DF_RESID) return;
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

// The same update in difference form, for a step d of the size of the iterate (the
// first refinement step from zero, where R = B - L(d) cancels to ~1e-5 of B):
//
//   t-pass  (d T^T)_b = rowsum(T)_b d_b + sum_{l != K} T_bl (d_{b+l-K} - d_b),
//   s-pass  likewise over rows for the terms whose s-factor is a stiffness or a
//           derivative (terms 0, 3, 4 of the five-term operator; 0, 4..7 of the
//           eight-term one), plain for the mass-like ones,
//   term 0  (K_s[h] + gamma M_s[h]) (x) M_t split exactly as d M_t^T = D (d + d N^T),
//           D = diag(rowsum M_t), N = D^{-1}(M_t - D): the s-pass acts on the exact
//           input d and on the small W' = d N^T, and the sum is scaled by D_b,
//
// with the row sums exact (double-float of the TwoSum of the FP64 coefficients) and
// the differences of the exact input taken exactly.  No rounding that the
// stiffness factors amplify by ~(mesh size)^-2 is then larger than the differences
// themselves: the evaluation error is ~2^-48 q of ||L(d)|| (about 1e-12 at q = 2047,
// against ~u q^2 / pi^2 = 4.7e-11 for an FP64 evaluation that rounds the t-pass
// mass product).  Tables: the difference-form double-float planes Sdd, Tdd.
template <int K, int NT>
__global__ void __launch_bounds__(DTB, 3) k_resid_dfd(DfArgs a) {
    using G = DGeo<K>;
    constexpr int P = G::P, TA = G::TA, HR = G::HR, WC = G::WC, NTP = NT * P;
    constexpr unsigned DM = NT == 5 ? 0x19u : 0xF1u;
    static_assert(DM & 1u, "term 0 runs its s-pass in difference form");
    extern __shared__ __align__(16) float dsm[];
    float* xh = dsm;                     // [HR][WC]
    float* xl = xh + HR * WC;            // [HR][WC]
    float* s_h = xl + HR * WC;           // [TA][NTP]
    float* s_l = s_h + TA * NTP;         // [TA][NTP]
    __shared__ double red[DTB / 32];
    const int tid = threadIdx.x, inst = blockIdx.z;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * DTB;
    const int q = a.q;
    {
        const float* dh = a.dh + (size_t)inst * a.bs;
        const float* dl = a.dl + (size_t)inst * a.bs;
        for (int r = tid / 32; r < HR; r += DTB / 32) {
            const int gr = a0 - K + r;
            const bool rok = gr >= 0 && gr < q;
            for (int cc = tid & 31; cc < WC; cc += 32) {
                const int gc = b0 - K + cc;
                float vh = 0.f, vl = 0.f;
                if (rok && gc >= 0 && gc < q) {
                    const size_t o = (size_t)gr * a.ld + gc;
                    vh = dh[o];
                    vl = dl[o];
                }
                xh[r * WC + cc] = vh;
                xl[r * WC + cc] = vl;
            }
        }
    }
    for (int idx = tid; idx < TA * NTP; idx += DTB) {
        const int e = idx / TA, r = idx - e * TA;
        const int gr = a0 + r;
        float vh = 0.f, vl = 0.f;
        if (gr < q) {
            const size_t o = (size_t)inst * a.s_bs + (size_t)e * q + gr;
            vh = a.Sh[o];
            vl = a.Sl[o];
        }
        s_h[r * NTP + e] = vh;
        s_l[r * NTP + e] = vl;
    }
    const int b = b0 + tid;
    float th[NT][P], tl[NT][P];   // term 0: N off the diagonal slot, D on it; others: row sum on it
#pragma unroll
    for (int i = 0; i < NT; ++i)
#pragma unroll
        for (int l = 0; l < P; ++l) {
            const size_t o = (size_t)(i * P + l) * q + b;
            th[i][l] = b < q ? a.Th[o] : 0.f;
            tl[i][l] = b < q ? a.Tl[o] : 0.f;
        }
    __syncthreads();
    // ring[i][j]: t-pass value of term i (term 0: W') for input row al + j; xr[j]: the
    // exact input of that row (term 0's s-pass operand)
    dfl ring[NT][P];
    dfl xr[P];
    auto tpass = [&](int lr, int slot) {
        const float* rh = xh + lr * WC + tid;
        const float* rl = xl + lr * WC + tid;
        const dfl xc{rh[K], rl[K]};
        dfl dx[P];
#pragma unroll
        for (int l = 0; l < P; ++l)
            if (l != K) dx[l] = sub_exact(dfl{rh[l], rl[l]}, xc);
        xr[slot] = xc;
        {
            dfl w = first_prod(th[0][0], tl[0][0], dx[0].h, dx[0].l);   // K >= 1: slot 0 is off the diagonal
#pragma unroll
            for (int l = 1; l < P; ++l)
                if (l != K) acc_prod(w, th[0][l], tl[0][l], dx[l].h, dx[l].l);
            ring[0][slot] = renorm(w);
        }
#pragma unroll
        for (int i = 1; i < NT; ++i) {
            dfl w = first_prod(th[i][K], tl[i][K], xc.h, xc.l);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) acc_prod(w, th[i][l], tl[i][l], dx[l].h, dx[l].l);
            ring[i][slot] = renorm(w);
        }
    };
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) tpass(r, r + 1);
    float rs = 0.f;
    double* Rg = a.R + (size_t)inst * a.bs;
#pragma unroll 1
    for (int al = 0; al < TA; ++al) {
        const int gr = a0 + al;
        const bool out = gr < q && b < q;
        const size_t o = (size_t)gr * a.ld + b;
        const double rold = out ? Rg[o] : 0.0;
#pragma unroll
        for (int j = 0; j + 1 < P; ++j) {
            xr[j] = xr[j + 1];
#pragma unroll
            for (int i = 0; i < NT; ++i) ring[i][j] = ring[i][j + 1];
        }
        tpass(al + 2 * K, P - 1);
        const float* ch = s_h + al * NTP;
        const float* cl = s_l + al * NTP;
        // term 0: D_b (S0-pass of d + S0-pass of W')
        dfl ya = first_prod(ch[K], cl[K], xr[K].h, xr[K].l);
        dfl yb = first_prod(ch[K], cl[K], ring[0][K].h, ring[0][K].l);
#pragma unroll
        for (int j = 0; j < P; ++j)
            if (j != K) {
                const dfl da = sub_exact(xr[j], xr[K]);
                const dfl db = sub_df(ring[0][j], ring[0][K]);
                acc_prod(ya, ch[j], cl[j], da.h, da.l);
                acc_prod(yb, ch[j], cl[j], db.h, db.l);
            }
        ya = renorm(ya);
        yb = renorm(yb);
        dfl sab;
        {
            float r;
            two_sum(ya.h, yb.h, sab.h, r);
            sab.l = (r + ya.l) + yb.l;
            sab = renorm(sab);
        }
        dfl y = first_prod(th[0][K], tl[0][K], sab.h, sab.l);
#pragma unroll
        for (int i = 1; i < NT; ++i) {
            dfl yi;
            if ((DM >> i) & 1u) {
                const dfl c = ring[i][K];
                yi = first_prod(ch[i * P + K], cl[i * P + K], c.h, c.l);
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (j != K) {
                        const dfl dv = sub_df(ring[i][j], c);
                        acc_prod(yi, ch[i * P + j], cl[i * P + j], dv.h, dv.l);
                    }
            } else {
                yi = first_prod(ch[i * P], cl[i * P], ring[i][0].h, ring[i][0].l);
#pragma unroll
                for (int j = 1; j < P; ++j) acc_prod(yi, ch[i * P + j], cl[i * P + j], ring[i][j].h, ring[i][j].l);
            }
            acc_df(y, renorm(yi));
        }
        if (out) {
            const double r = rold - ((double)y.h + (double)y.l);
            Rg[o] = r;
            const float rf = (float)r;
            rs = fmaf(rf, rf, rs);
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

template <int K, int NT>
mofem_status launch_dfd_t(const DfArgs& a, int batch, int* nblk, cudaStream_t st) {
    using G = DGeo<K>;
    const size_t smem = sizeof(float) * (2 * (size_t)G::HR * G::WC + 2 * (size_t)G::TA * NT * G::P);
    static std::atomic<bool> attr[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(k_resid_dfd<K, NT>, (int)smem, attr));
    dim3 grid((a.q + DTB - 1) / DTB, (a.q + G::TA - 1) / G::TA, batch);
    if (nblk) *nblk = grid.x * grid.y;
    k_resid_dfd<K, NT><<<grid, DTB, smem, st>>>(a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

template <int K, int NT, int MODE = DF_RESID>
mofem_status launch_df_t(const DfArgs& a, int batch, int* nblk, cudaStream_t st) {
    using G = DGeo<K>;
    const size_t smem = sizeof(float) * (2 * (size_t)G::HR * G::WC + 2 * (size_t)G::TA * NT * G::P);
    static std::atomic<bool> attr[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(k_resid_df<K, NT, MODE>, (int)smem, attr));
    dim3 grid((a.q + DTB - 1) / DTB, (a.q + G::TA - 1) / G::TA, batch);
    if (nblk) *nblk = grid.x * grid.y;
    k_resid_df<K, NT, MODE><<<grid, DTB, smem, st>>>(a);
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
    return ((q + DTB - 1) / DTB) * ((q + DGeo<1>::TA - 1) / DGeo<1>::TA);
}

// Forms served: the ring and the T coefficients in registers (NT * (2K+1) <= 40,
// as the packed FP32 apply); others return MOFEM_ERR_UNSUPPORTED and the caller
// recomputes the residual in FP64.
mofem_status launch_residual_update_df(const mofem_ctx* c, const float* dh, const float* dl, double* R,
                                       double* partial, int* nblk, cudaStream_t st) {
    if (c->NT * (2 * c->K + 1) > 40 || !c->Sdf || !c->Tdf) return MOFEM_ERR_UNSUPPORTED;
    DfArgs a{};
    a.dh = dh; a.dl = dl;
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

bool residual_update_dfd_ok(const mofem_ctx* c) {
    if (!c->Sdd || !c->Tdd) return false;
    return (c->K == 2 && c->NT == 5) || (c->K == 1 && (c->NT == 5 || c->NT == 8));
}

// Forms served: K = 1 (five or eight terms) and K = 2 (five terms), with the ring and the
// T coefficients in registers; others return MOFEM_ERR_UNSUPPORTED and the caller
// recomputes the residual in FP64.
mofem_status launch_residual_update_dfd(const mofem_ctx* c, const float* dh, const float* dl, double* R,
                                        double* partial, int* nblk, cudaStream_t st) {
    if (!residual_update_dfd_ok(c)) return MOFEM_ERR_UNSUPPORTED;
    DfArgs a{};
    a.dh = dh; a.dl = dl;
    const long long sp = (long long)c->batch * c->NT * c->P * c->q;
    const long long tp = (long long)c->NT * c->P * c->q;
    a.Sh = c->Sdd; a.Sl = c->Sdd + sp; a.s_bs = (long long)c->NT * c->P * c->q;
    a.Th = c->Tdd; a.Tl = c->Tdd + tp;
    a.R = R; a.bs = (long long)c->q * c->ld; a.ld = c->ld; a.q = c->q;
    a.partial = partial;
    if (c->K == 2) return launch_dfd_t<2, 5>(a, c->batch, nblk, st);
    if (c->NT == 8) return launch_dfd_t<1, 8>(a, c->batch, nblk, st);
    return launch_dfd_t<1, 5>(a, c->batch, nblk, st);
}

mofem_status launch_rhs_df(const mofem_ctx* c, const double* F, double* B, long long b_bs, int b_ld, cudaStream_t st) {
    if (!c->Srdf || !c->Trdf || c->K < 1 || c->K > 4) return MOFEM_ERR_UNSUPPORTED;
    DfArgs a{};
    a.X = F; a.x_bs = (long long)c->n * c->n; a.x_ld = c->n;
    a.rows_in = a.cols_in = c->n; a.off = c->off;
    a.Y = B; a.y_bs = b_bs; a.y_ld = b_ld;
    const long long sp = (long long)c->batch * c->P * c->q, tp = (long long)c->P * c->q;
    a.Sh = c->Srdf; a.Sl = c->Srdf + sp; a.s_bs = (long long)c->P * c->q;
    a.Th = c->Trdf; a.Tl = c->Trdf + tp;
    a.q = c->q;
    switch (c->K) {
        case 1: return launch_df_t<1, 1, DF_APPLY64>(a, c->batch, nullptr, st);
        case 2: return launch_df_t<2, 1, DF_APPLY64>(a, c->batch, nullptr, st);
        case 3: return launch_df_t<3, 1, DF_APPLY64>(a, c->batch, nullptr, st);
        default: return launch_df_t<4, 1, DF_APPLY64>(a, c->batch, nullptr, st);
    }
}
