// Packed-FP32 PCG form of the banded multiterm operator apply (Sec. 5, operator
// L~ of the multiterm Sylvester equation), the FP32 operator of the mixed inner
// solve.  Same arithmetic as compute_tile<float> (difference form, exact mass
// split of term 0), restructured for the sm_100-family paired FP32 pipe and for
// streaming:
//
//   * each thread owns two adjacent columns b, b+1 and every product, sum and
//     fused multiply-add acts on the pair at once (one f32x2 instruction per two
//     results), which halves the instruction count of the t- and s-passes;
//   * a CTA is 64 threads = 64 column pairs (a strip of 128 columns) and streams
//     down a long segment of rows of one instance (grid: strips x segments x
//     instances, sized to one wave of resident CTAs), with a register ring of the
//     last 2K+1 t-pass rows (compile-time slots after unrolling by 2K+1): the
//     T coefficients are loaded once per segment and only 2K halo rows per
//     segment are recomputed;
//   * Z, Q_prev and the segment's S rows arrive by TMA in chunks of CR rows into a
//     ring of D chunks (one mbarrier per slot, bounded waits); a chunk slot is
//     refilled CR * D rows ahead once every thread has passed its last row, so the
//     loads overlap the arithmetic of the rows before them; the search direction
//     X = Z + beta Q_prev is formed on the fly from both staged rows and the owned
//     rows of the new direction are written from registers;
//   * the s-pass coefficients come from a copy of the S tables laid out per row
//     with every coefficient duplicated into both lanes of a float2, so a
//     shared-memory broadcast feeds a paired FMA directly.
//
// Fused epilogue: per-CTA FP64 partials of <X, L(X)> and <L(X), Z> and, in the
// last CTA of each instance, alpha = <R, Z> / <Q, L(Q)> and the flexible-beta
// numerator term <R_new, Z> = <R, Z> - alpha <L(Q), Z> (fixed-order sums of the
// partials), so the residual update never reads Z again.
#pragma once
#include "apply_impl.cuh"

namespace mofem_apply_impl {

template <int K, int NT>
struct Geo3 {
    static constexpr int P = 2 * K + 1;
    static constexpr int NTH = 64;                       // threads = column pairs per CTA
    static constexpr int CR = 4;                         // rows per staged chunk
    static constexpr int D = 4;                          // chunks in the ring
    static constexpr int RING = CR * D;                  // staged rows (power of two)
    static constexpr int SR2 = ((NT * P + 3) / 4) * 4;   // float2 per duplicated S row (a chunk of S rows
                                                         // stays a 128-byte multiple)
    static constexpr bool TREG = NT * P <= 25;           // T coefficients in registers, else shared
    static constexpr int KE = K + (K & 1);               // left reach rounded to an even column
    static constexpr int ZCH = CR * WCT;                 // floats per chunk of Z (and of Q_prev)
    static constexpr int SCH = CR * SR2;                 // float2 per chunk of S rows
    static constexpr uint32_t CHUNK_BYTES = 2u * ZCH * 4u + (uint32_t)SCH * 8u;
    static constexpr size_t SMEM = (size_t)D * CHUNK_BYTES + (TREG ? 0 : (size_t)NT * P * NTH * 8) + 128;
    // register budget: 6 resident CTAs (168 registers) with T in registers; with T in shared
    // memory the staging caps residency lower, which leaves room for the longer ring
    static constexpr int MINB = TREG ? 6 : 4;
    static_assert((RING & (RING - 1)) == 0, "ring rows must be a power of two");
    static_assert((ZCH * 4) % 128 == 0 && (SCH * 8) % 128 == 0, "TMA destinations stay 128-byte aligned");
    // a chunk is refilled only after its last row is done; the rows that wait for it must
    // not be the ones that release it: (D - 1) CR >= 2K (t-pass reach) + 2K (unrolled block)
    static_assert((D - 1) * CR >= 4 * K, "ring too short for the stencil reach");
};

// Operator forms served by the packed kernel (the ring and, if TREG, the T
// coefficients live in registers); the others use k_apply_pcg.
__host__ __device__ constexpr bool packed_apply_ok(int K, int NT) { return NT * (2 * K + 1) <= 40; }

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - c, one rounding (fma with an exact -1 product)
__device__ __forceinline__ float2 f2sub(float2 a, float2 c) { return __ffma2_rn(c, make_float2(-1.f, -1.f), a); }

// Rows of one segment and the number of segments per strip: at most one wave of resident
// CTAs over all strips and instances (a partial second wave would double the time of the
// SMs that run it), at least 8 (2K + 8) rows per segment.
__host__ __device__ inline int apply3_segments(int q, int strips, int batch, int ctas_wanted, int K) {
    const int min_rows = 8 * (2 * K + 8);
    int segs = ctas_wanted / (strips * batch);
    const int max_segs = (q + min_rows - 1) / min_rows;
    if (segs > max_segs) segs = max_segs;
    return segs < 1 ? 1 : segs;
}

template <int K, int NT>
__global__ void __launch_bounds__(Geo3<K, NT>::NTH, Geo3<K, NT>::MINB)
    k_apply_pcg3(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mQ,
                 const __grid_constant__ CUtensorMap mS, ApplyPcgArgs a, int seg_rows) {
    using G = Geo3<K, NT>;
    constexpr int P = G::P, SR2 = G::SR2, KE = G::KE, CR = G::CR, D = G::D, RING = G::RING, NTH = G::NTH;
    constexpr unsigned DM = DiffMask<NT>::value;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    float* Zs = reinterpret_cast<float*>(sbase);               // [RING][WCT]
    float* Qs = Zs + RING * WCT;                                // [RING][WCT]
    float2* S2s = reinterpret_cast<float2*>(Qs + RING * WCT);   // [RING][SR2]
    float2* T2s = S2s + RING * SR2;                             // [NT*P][NTH] (!TREG)
    __shared__ __align__(8) unsigned long long bar[D];
    __shared__ double red[NTH / 32];
    __shared__ float beta_s;
    __shared__ int fail_s, last_s;
    const int tid = threadIdx.x, inst = blockIdx.z;
    PcgScalars* sc = a.sc + inst;
    if (a.use_sc && !sc->active) return;
    const int b0 = blockIdx.x * TB;
    const int a_lo = blockIdx.y * seg_rows;
    const int L = max(0, min(a.q, a_lo + seg_rows) - a_lo);   // output rows of this segment
    // rows are computed in whole blocks of P (straight-line code, stores guarded): the
    // last block may run past L into zero-filled or neighbouring rows, never stored
    const int nblk_rows = (L + P - 1) / P;
    const int LP = nblk_rows * P;
    const int nch = (LP + 2 * K + CR - 1) / CR;                 // chunks of input rows a_lo - K ...
    if (tid == 0) {
        for (int i = 0; i < D; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        beta_s = (a.use_sc && sc->iters > 0) ? (float)sc->beta : 0.f;
    }
    __syncthreads();
    // chunk c -> ring slot c % D: input rows a_lo - K + c CR .. (Z, Q_prev) and S rows a_lo + c CR ..
    auto issue = [&](int c) {
        const int slot = c % D;
        const uint32_t b = smem_u32(&bar[slot]);
        const uint64_t pz = reinterpret_cast<uint64_t>(&mZ), pq = reinterpret_cast<uint64_t>(&mQ),
                       ps = reinterpret_cast<uint64_t>(&mS);
        const int x0 = b0 - XPAD, y0 = a_lo - K + c * CR;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(G::CHUNK_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(S2s + slot * G::SCH)), "l"(ps), "r"(b), "r"(0), "r"(a_lo + c * CR), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Zs + slot * G::ZCH)), "l"(pz), "r"(b), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Qs + slot * G::ZCH)), "l"(pq), "r"(b), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
    };
    if (tid == 0)
        for (int c = 0; c < D && c < nch; ++c) issue(c);
    const int cp = tid;
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
        for (int idx = tid; idx < NT * P * NTH; idx += NTH) {
            const int il = idx / NTH, c = idx - il * NTH;
            const int bb = b0 + 2 * c;
            const size_t o = (size_t)il * a.q + bb;
            T2s[idx] = make_float2(bb < a.q ? Tt[o] : 0.f, bb + 1 < a.q ? Tt[o + 1] : 0.f);
        }
        __syncthreads();
    }
    auto tcoef = [&](int i, int l) -> float2 {
        if constexpr (G::TREG) return tc[i][l];
        else return T2s[(i * P + l) * NTH + cp];
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
    bool failed = false;
    int waited = 0, released = 0;
    auto wait_upto = [&](int need) {   // chunks 0 .. need-1 resident
        while (waited < need) {
            if (!failed) failed = !mbar_wait_bounded(smem_u32(&bar[waited % D]), (uint32_t)((waited / D) & 1));
            ++waited;
        }
    };
    float2 ring[NT][P];
    float2 xr0[P];
    // t-pass of input index i (input row a_lo - K + i) into ring slot `slot`
    auto tpass = [&](int i, int slot) {
        const int rr = (i & (RING - 1)) * WCT + XPAD + 2 * cp - KE;
        const float2* z2 = reinterpret_cast<const float2*>(Zs + rr);
        const float2* q2 = reinterpret_cast<const float2*>(Qs + rr);
        float xs[2 * KE + 2];
#pragma unroll
        for (int m = 0; m <= KE; ++m) {
            const float2 v = f2fma(beta2, q2[m], z2[m]);
            xs[2 * m] = v.x;
            xs[2 * m + 1] = v.y;
        }
        const float2 xc = make_float2(xs[KE], xs[KE + 1]);
        xr0[slot] = xc;
        const int orow = i - K;   // segment output row whose centre this is
        if (orow >= 0 && orow < L && col_ok)
            *reinterpret_cast<float2*>(Qn + (size_t)(a_lo + orow) * a.ld + b) = xc;
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
        for (int t = 1; t < NT; ++t) {
            float2 w = f2mul(tcoef(t, K), xc);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = f2fma(tcoef(t, l), d[l], w);
            ring[t][slot] = w;
        }
    };
    wait_upto(min(nch, (2 * K - 1) / CR + 1));
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) tpass(r, r);
    float2 acc = make_float2(0.f, 0.f), acz = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int m = 0; m < nblk_rows; ++m) {
        const int j0 = m * P;
        const int jend = j0 + P;
        wait_upto(min(nch, (jend - 1 + 2 * K) / CR + 1));
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int j = j0 + u;   // segment output row
            {
                tpass(j + 2 * K, (u + P - 1) % P);
                // row coefficients as 16-byte broadcasts: float4 e/2 holds coefficients e, e+1 (SR2 even)
                const float4* srow4 = reinterpret_cast<const float4*>(S2s + (j & (RING - 1)) * SR2);
                auto sc2 = [&](int e) -> float2 {
                    const float4 v = srow4[e >> 1];
                    return (e & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                };
                float2 yt[NT];
                {
                    const float2 xc = xr0[(u + K) % P], wc = ring[0][(u + K) % P];
                    float2 ya = f2mul(sc2(K), xc), yb = f2mul(sc2(K), wc);
#pragma unroll
                    for (int jj = 0; jj < P; ++jj)
                        if (jj != K) {
                            ya = f2fma(sc2(jj), f2sub(xr0[(u + jj) % P], xc), ya);
                            yb = f2fma(sc2(jj), f2sub(ring[0][(u + jj) % P], wc), yb);
                        }
                    yt[0] = f2mul(d0, f2add(ya, yb));
                }
#pragma unroll
                for (int t = 1; t < NT; ++t) {
                    const float2 wc = ring[t][(u + K) % P];
                    float2 y = f2mul(sc2(t * P + K), wc);
#pragma unroll
                    for (int jj = 0; jj < P; ++jj)
                        if (jj != K) {
                            if ((DM >> t) & 1u) y = f2fma(sc2(t * P + jj), f2sub(ring[t][(u + jj) % P], wc), y);
                            else y = f2fma(sc2(t * P + jj), ring[t][(u + jj) % P], y);
                        }
                    yt[t] = y;
                }
                // pairwise sum of the term results (independent chains above)
#pragma unroll
                for (int s = 1; s < NT; s *= 2)
#pragma unroll
                    for (int t = 0; t + s < NT; t += 2 * s) yt[t] = f2add(yt[t], yt[t + s]);
                const float2 y = yt[0];
                if (col_ok && j < L) {
                    *reinterpret_cast<float2*>(LQ + (size_t)(a_lo + j) * a.ld + b) = y;
                    acc = f2fma(xr0[(u + K) % P], y, acc);
                    const float2 zc = *reinterpret_cast<const float2*>(
                        Zs + ((j + K) & (RING - 1)) * WCT + XPAD + 2 * cp);
                    acz = f2fma(zc, y, acz);
                }
            }
        }
        // chunks whose last row (its S rows end at output row (c + 1) CR - 1) is done: refill
        const int can = min(nch, jend / CR);
        if (can > released) {
            __syncthreads();   // every thread is past the rows of those slots
            if (tid == 0)
                for (int c = released; c < can; ++c)
                    if (c + D < nch) issue(c + D);
            released = can;
        }
    }
    wait_upto(nch);   // every issued copy has landed before the CTA exits
    if (failed) atomicOr(&fail_s, 1);
    double s = block_sum<NTH>((double)acc.x + (double)acc.y, red);
    __syncthreads();   // red[] is reused
    const double s2 = a.partial2 ? block_sum<NTH>((double)acz.x + (double)acz.y, red) : 0.0;
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

// Resident CTAs of the streaming apply on the current device (one wave), per (K, NT).
template <int K, int NT>
int apply3_ctas_wanted_t() {
    using G = Geo3<K, NT>;
    static std::atomic<int> cache[MOFEM_MAX_DEV];
    const int slot = dev_slot();
    int n = cache[slot].load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
        smem_attr_once(k_apply_pcg3<K, NT>, (int)G::SMEM, attr_done);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_pcg3<K, NT>, G::NTH, G::SMEM) !=
                cudaSuccess ||
            per < 1)
            per = 1;
        n = (sms > 0 ? sms : 1) * per;
        cache[slot].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int K, int NT>
mofem_status launch_pcg3_t(const CUtensorMap& mZ, const CUtensorMap& mQ, const CUtensorMap& mS,
                           const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    using G = Geo3<K, NT>;
    auto kern = k_apply_pcg3<K, NT>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)G::SMEM, attr_done));
    const int strips = (a.q + TB - 1) / TB;
    const int segs = apply3_segments(a.q, strips, batch, apply3_ctas_wanted_t<K, NT>(), K);
    constexpr int P = 2 * K + 1;   // segments of whole row blocks: only the last one is ragged
    const int seg_rows = ((a.q + segs - 1) / segs + P - 1) / P * P;
    dim3 grid(strips, segs, batch);
    kern<<<grid, G::NTH, G::SMEM, st>>>(mZ, mQ, mS, a, seg_rows);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
