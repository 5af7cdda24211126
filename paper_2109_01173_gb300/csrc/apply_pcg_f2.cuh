// Packed-FP32 PCG form of the banded multiterm operator apply (Sec. 5, operator
// L~ of the multiterm Sylvester equation), the FP32 operator of the mixed inner
// solve.  Same arithmetic as compute_tile<float> (difference form, exact mass
// split of term 0), restructured for the sm_100-family paired FP32 pipe:
//
//   * each thread owns two adjacent columns b, b+1 and every product, sum and
//     fused multiply-add acts on the pair at once (one f32x2 instruction per two
//     results), which halves the instruction count of the t- and s-passes;
//   * the CTA is 128 columns x TA rows, 128 threads = 64 column pairs x 2 row
//     groups; each group streams down its own TA/2 output rows with a register
//     ring of the last 2K+1 t-pass rows (compile-time slots after unrolling);
//   * Z and Q_prev arrive by TMA as one box each (the tile with its K-row halo)
//     together with the tile's S rows, all on one mbarrier waited once (a
//     per-row wait on 4-row chunks measured 4% slower: overlap between the 3
//     resident CTAs of an SM hides the load better than overlap within one); the
//     search direction X = Z + beta Q_prev is formed on the fly from both staged
//     tiles and the owned rows of the new direction are written from registers;
//   * the s-pass coefficients arrive by TMA as well, from a copy of the S tables
//     laid out per row with every coefficient duplicated into both lanes of a
//     float2, so a shared-memory broadcast feeds a paired FMA directly.
//
// Fused epilogue: per-CTA FP64 partials of <X, L(X)> and <L(X), Z> and, in the
// last CTA of each instance, alpha = <R, Z> / <Q, L(Q)> and the flexible-beta
// numerator term <R_new, Z> = <R, Z> - alpha <L(Q), Z> (fixed-order sums of the
// partials), so the residual update never reads Z again.
#pragma once
#include "apply_impl.cuh"

namespace mofem_apply_impl {

#ifndef MOFEM_APPLY_ROWS
#define MOFEM_APPLY_ROWS 20   // target output rows per row group (rounded up to whole ring periods)
#endif
#ifndef MOFEM_APPLY_MINB
#define MOFEM_APPLY_MINB 3    // resident CTAs per SM the register budget is sized for
#endif

template <int K, int NT>
struct Geo2 {
    static constexpr int P = 2 * K + 1;
    static constexpr int NPAIR = TB / 2;                 // column pairs per CTA
    static constexpr int RG = 2;                         // row groups
    static constexpr int NTH = NPAIR * RG;               // threads per CTA
    static constexpr int MRG = (MOFEM_APPLY_ROWS + P - 1) / P;   // ring periods per group
    static constexpr int TAG = MRG * P;                  // output rows per group
    static constexpr int TA = RG * TAG;                  // output rows per CTA
    static constexpr int HR = TA + 2 * K;                // staged rows
    static constexpr int ROWS = (HR + 3) / 4 * 4;        // staging rows (4 x 544 B: 128-byte multiple)
    static constexpr int ZBUF = ROWS * WCT;              // floats per staging buffer
    static constexpr int SR2 = ((NT * P + 1) / 2) * 2;   // float2 per duplicated S row (16-byte rows)
    static constexpr bool TREG = NT * P <= 25;           // T coefficients in registers, else shared
    static constexpr int KE = K + (K & 1);               // left reach rounded to an even column
    static constexpr size_t SMEM = (size_t)2 * ZBUF * 4 + (size_t)TA * SR2 * 8 +
                                   (TREG ? 0 : (size_t)NT * P * NPAIR * 8) + 128;
};

// Operator forms served by the packed kernel (the ring and, if TREG, the T
// coefficients live in registers); the others use k_apply_pcg.
__host__ __device__ constexpr bool packed_apply_ok(int K, int NT) { return NT * (2 * K + 1) <= 40; }

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - c, one rounding (fma with an exact -1 product)
__device__ __forceinline__ float2 f2sub(float2 a, float2 c) { return __ffma2_rn(c, make_float2(-1.f, -1.f), a); }

template <int K, int NT>
__global__ void __launch_bounds__(Geo2<K, NT>::NTH, MOFEM_APPLY_MINB)
    k_apply_pcg2(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mQ,
                 const __grid_constant__ CUtensorMap mS, ApplyPcgArgs a) {
    using G = Geo2<K, NT>;
    constexpr int P = G::P, TAG = G::TAG, TA = G::TA, HR = G::HR, SR2 = G::SR2, KE = G::KE;
    constexpr int NPAIR = G::NPAIR, MRG = G::MRG;
    constexpr unsigned DM = DiffMask<NT>::value;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    float* Zs = reinterpret_cast<float*>(sbase);               // [ROWS][WCT]
    float* Qs = Zs + G::ZBUF;                                   // [ROWS][WCT]
    float2* S2s = reinterpret_cast<float2*>(Qs + G::ZBUF);      // [TA][SR2]
    float2* T2s = S2s + TA * SR2;                               // [NT*P][NPAIR] (!TREG)
    __shared__ __align__(8) unsigned long long bar;
    __shared__ double red[G::NTH / 32];
    __shared__ float beta_s;
    __shared__ int fail_s, last_s;
    const int tid = threadIdx.x, inst = blockIdx.z;
    PcgScalars* sc = a.sc + inst;
    if (a.use_sc && !sc->active) return;
    const int a0 = blockIdx.y * TA, b0 = blockIdx.x * TB;
    const uint32_t bar0 = smem_u32(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        beta_s = (a.use_sc && sc->iters > 0) ? (float)sc->beta : 0.f;
    }
    __syncthreads();
    if (tid == 0) {
        const uint64_t pz = reinterpret_cast<uint64_t>(&mZ), pq = reinterpret_cast<uint64_t>(&mQ),
                       ps = reinterpret_cast<uint64_t>(&mS);
        const int x0 = b0 - XPAD, y0 = a0 - K;
        const uint32_t bytes = 2u * HR * WCT * 4u + (uint32_t)(TA * SR2 * 8);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar0), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(S2s)), "l"(ps), "r"(bar0), "r"(0), "r"(a0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Zs)), "l"(pz), "r"(bar0), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Qs)), "l"(pq), "r"(bar0), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
    }
    const int cp = tid % NPAIR, grp = tid / NPAIR;
    const int b = b0 + 2 * cp;
    const float* Tt = reinterpret_cast<const float*>(a.T);
    auto tload = [&](int il) -> float2 {
        const size_t o = (size_t)il * a.q + b;
        return make_float2(b < a.q ? Tt[o] : 0.f, b + 1 < a.q ? Tt[o + 1] : 0.f);
    };
    float2 tc[G::TREG ? NT : 1][G::TREG ? P : 1];
    if constexpr (G::TREG) {
#pragma unroll
        for (int i = 0; i < NT; ++i)
#pragma unroll
            for (int l = 0; l < P; ++l) tc[i][l] = tload(i * P + l);
    } else {
        for (int idx = tid; idx < NT * P * NPAIR; idx += G::NTH) {
            const int il = idx / NPAIR, c = idx - il * NPAIR;
            const int bb = b0 + 2 * c;
            const size_t o = (size_t)il * a.q + bb;
            T2s[idx] = make_float2(bb < a.q ? Tt[o] : 0.f, bb + 1 < a.q ? Tt[o + 1] : 0.f);
        }
        __syncthreads();
    }
    auto tcoef = [&](int i, int l) -> float2 {
        if constexpr (G::TREG) return tc[i][l];
        else return T2s[(i * P + l) * NPAIR + cp];
    };
    // Term 0 exact mass split: X M_t^T = D (X + X N^T), N = D^{-1}(M_t - D) (zero row sums).
    const float2 d0 = tcoef(0, K);
    float2 n0[P];
    {
        const float2 dinv = make_float2(d0.x != 0.f ? 1.f / d0.x : 0.f, d0.y != 0.f ? 1.f / d0.y : 0.f);
#pragma unroll
        for (int l = 0; l < P; ++l) n0[l] = (l == K) ? make_float2(0.f, 0.f) : f2mul(tcoef(0, l), dinv);
    }
    const float bsc = beta_s;
    const float2 beta2 = make_float2(bsc, bsc);
    float* Qn = reinterpret_cast<float*>(a.Qnew) + (size_t)inst * a.bs;
    float* LQ = reinterpret_cast<float*>(a.LQ) + (size_t)inst * a.bs;
    const bool col_ok = b < a.ld;   // pad columns [q, ld) receive zeros
    const int lr0 = grp * TAG;      // first staged row of this group's window
    const bool failed = !mbar_wait_bounded(bar0, 0);   // the whole tile, its halo and the S rows
    float2 ring[NT][P];
    float2 xr0[P];
    auto tpass = [&](int lr, int slot) {
        const float2* z2 = reinterpret_cast<const float2*>(Zs + lr * WCT + XPAD + 2 * cp - KE);
        const float2* q2 = reinterpret_cast<const float2*>(Qs + lr * WCT + XPAD + 2 * cp - KE);
        float xs[2 * KE + 2];
#pragma unroll
        for (int m = 0; m <= KE; ++m) {
            const float2 v = f2fma(beta2, q2[m], z2[m]);
            xs[2 * m] = v.x;
            xs[2 * m + 1] = v.y;
        }
        const float2 xc = make_float2(xs[KE], xs[KE + 1]);
        xr0[slot] = xc;
        const int orow = lr - K - lr0;   // group-local output row whose centre this is
        if (orow >= 0 && orow < TAG) {
            const int gr = a0 + lr - K;
            if (gr < a.q && col_ok) *reinterpret_cast<float2*>(Qn + (size_t)gr * a.ld + b) = xc;
        }
        float2 d[P];
#pragma unroll
        for (int l = 0; l < P; ++l)
            if (l != K) d[l] = f2sub(make_float2(xs[KE + l - K], xs[KE + l - K + 1]), xc);
        {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = f2fma(n0[l], d[l], w);
            ring[0][slot] = w;
        }
#pragma unroll
        for (int i = 1; i < NT; ++i) {
            float2 w = f2mul(tcoef(i, K), xc);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = f2fma(tcoef(i, l), d[l], w);
            ring[i][slot] = w;
        }
    };
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) tpass(lr0 + r, r);
    float2 acc = make_float2(0.f, 0.f), acz = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int m = 0; m < MRG; ++m) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int al = lr0 + m * P + u;   // tile-local output row
            tpass(al + 2 * K, (u + P - 1) % P);
            // row coefficients as 16-byte broadcasts: float4 e/2 holds coefficients e, e+1 (SR2 even)
            const float4* srow4 = reinterpret_cast<const float4*>(S2s + al * SR2);
            auto sc2 = [&](int e) -> float2 {
                const float4 v = srow4[e >> 1];
                return (e & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
            };
            float2 yt[NT];
            {
                const float2 xc = xr0[(u + K) % P], wc = ring[0][(u + K) % P];
                float2 ya = f2mul(sc2(K), xc), yb = f2mul(sc2(K), wc);
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (j != K) {
                        ya = f2fma(sc2(j), f2sub(xr0[(u + j) % P], xc), ya);
                        yb = f2fma(sc2(j), f2sub(ring[0][(u + j) % P], wc), yb);
                    }
                yt[0] = f2mul(d0, f2add(ya, yb));
            }
#pragma unroll
            for (int i = 1; i < NT; ++i) {
                const float2 wc = ring[i][(u + K) % P];
                float2 y = f2mul(sc2(i * P + K), wc);
#pragma unroll
                for (int j = 0; j < P; ++j)
                    if (j != K) {
                        if ((DM >> i) & 1u) y = f2fma(sc2(i * P + j), f2sub(ring[i][(u + j) % P], wc), y);
                        else y = f2fma(sc2(i * P + j), ring[i][(u + j) % P], y);
                    }
                yt[i] = y;
            }
            // pairwise sum of the term results (independent chains above)
#pragma unroll
            for (int s = 1; s < NT; s *= 2)
#pragma unroll
                for (int i = 0; i + s < NT; i += 2 * s) yt[i] = f2add(yt[i], yt[i + s]);
            const float2 y = yt[0];
            const int gr = a0 + al;
            if (gr < a.q && col_ok) {
                *reinterpret_cast<float2*>(LQ + (size_t)gr * a.ld + b) = y;
                acc = f2fma(xr0[(u + K) % P], y, acc);
                acz = f2fma(*reinterpret_cast<const float2*>(Zs + (al + K) * WCT + XPAD + 2 * cp), y, acz);
            }
        }
    }
    if (failed) atomicOr(&fail_s, 1);
    double s = block_sum<G::NTH>((double)acc.x + (double)acc.y, red);
    __syncthreads();   // red[] is reused
    const double s2 = a.partial2 ? block_sum<G::NTH>((double)acz.x + (double)acz.y, red) : 0.0;
    const int nblk = gridDim.x * gridDim.y;
    if (tid == 0) {
        if (fail_s) atomicOr(a.status, DEV_ERR_TIMEOUT);
        a.partial[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s;
        if (a.partial2) a.partial2[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s2;
        __threadfence();
        const unsigned t = atomicAdd(a.counter + inst, 1u);
        last_s = (t == (unsigned)nblk - 1) ? 1 : 0;
    }
    __syncthreads();
    if (last_s && tid < 32) {
        __threadfence();
        const double qlq = warp_sum_partials(a.partial + (size_t)inst * nblk, nblk);
        const double lqz = a.partial2 ? warp_sum_partials(a.partial2 + (size_t)inst * nblk, nblk) : 0.0;
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
            if (a.partial2) sc->rzo = sc->rz - al * lqz;   // <R - alpha L(Q), Z>
        }
    }
}

template <int K, int NT>
mofem_status launch_pcg2_t(const CUtensorMap& mZ, const CUtensorMap& mQ, const CUtensorMap& mS,
                           const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    using G = Geo2<K, NT>;
    auto kern = k_apply_pcg2<K, NT>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)G::SMEM, attr_done));
    dim3 grid((a.q + TB - 1) / TB, (a.q + G::TA - 1) / G::TA, batch);
    kern<<<grid, G::NTH, G::SMEM, st>>>(mZ, mQ, mS, a);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
