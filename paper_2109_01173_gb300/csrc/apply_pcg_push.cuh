// Streaming packed-FP32 PCG-form apply with the s-pass in push form (Sec. 5, operator
// L~ of the multiterm Sylvester equation; the FP32 operator of the mixed inner solve).
//
// The t-pass is the one of k_apply_pcg3 (two adjacent columns per thread, paired FP32,
// difference form, exact mass split of term 0).  The s-pass is reorganised so that no
// window of t-pass rows has to stay in registers: when input row g has been through the
// t-pass, its contributions are added at once into the 2K + 1 output rows g - K .. g + K
// that it reaches, held in a register ring of accumulators; output row j is complete
// after input row j + K and is stored then.
//
//   plain terms:       y[j] += S[j][g] W[g]                           (j = g - K .. g + K)
//   difference terms:  y[j] = c_j W[j] + sum_{m != 0} S[j][j+m] (W[j+m] - W[j])
//                      (c_j the row sum) is rewritten over the consecutive differences
//                      delta[k] = W[k+1] - W[k], k = j - K .. j + K - 1:
//                        W[j+m] - W[j] = delta[j] + .. + delta[j+m-1]         (m > 0)
//                                      = -(delta[j+m] + .. + delta[j-1])      (m < 0)
//                      so that y[j] = c_j W[j] + sum_k a_j(k - j) delta[k] with
//                        a_j(d) =  sum_{m > d} S[j][j+m]   (d >= 0)
//                        a_j(d) = -sum_{m <= d} S[j][j+m]  (d < 0);
//                      input row g pushes delta[g-1] into rows g - K .. g + K - 1 and
//                      c_g W[g] into row g.
//
// Like the difference form of k_apply_pcg3 this never forms W[j+m] - W[j] sums of large
// cancelling terms: every product is a coefficient times a difference of neighbouring
// rows (one rounding each).  The coefficients of input row g (P per term: 2K partial
// sums and the row sum for difference terms, the matrix column S[g-K..g+K][g] for plain
// terms) are tabulated at setup in FP64 and rounded once; Z, Q_prev and those rows
// arrive by TMA in chunks of CR rows into a ring of D chunks, as in k_apply_pcg3.
//
// Registers per thread: the T coefficients, 3 (2K + 1) float2 (two accumulator rings and
// the ring of new-direction centres) and one float2 per difference term, against
// NT (2K + 2) + (2K + 2) float2 for the row window of k_apply_pcg3.
#pragma once
#include "apply_pcg_f2.cuh"

namespace mofem_apply_impl {

template <int K, int NT, int NS = 1>
struct Geo4 {
    static constexpr int P = 2 * K + 1;
    static constexpr int NTH = 64;                       // threads = column pairs per CTA
    static constexpr int CR = 4;                         // rows per staged chunk
    static constexpr int D = 4;                          // chunks in the ring
    static constexpr int RING = CR * D;                  // staged rows (power of two)
    static constexpr int SR = ((NT * P + 7) / 8) * 8;    // floats per coefficient row
    static constexpr int KE = K + (K & 1);               // left reach rounded to an even column
    static constexpr int ZCH = CR * WCT;                 // floats per chunk of Z (and of Q_prev)
    static constexpr int SCH = CR * SR;                  // floats per chunk of coefficient rows
    static constexpr uint32_t CHUNK_BYTES = 2u * ZCH * 4u + (uint32_t)SCH * 4u;
    static constexpr size_t SMEM = (size_t)NS * D * CHUNK_BYTES + 128;   // one ring per row stream
    // one stream: 128 registers (16 warps per SM) where they suffice; two: the shared memory of
    // five CTAs per SM
    static constexpr int MINB = NS == 1 ? (NT * P <= 25 ? 8 : 5) : 5;
    static_assert((RING & (RING - 1)) == 0, "ring rows must be a power of two");
    static_assert((ZCH * 4) % 128 == 0 && (SCH * 4) % 128 == 0, "TMA destinations stay 128-byte aligned");
    // one block of P input rows reads rows back to K before its first: those rows and the
    // block span at most D - 1 released-and-refilled chunk boundaries
    static_assert((D - 1) * CR >= P + K - 1, "ring too short for the block and its reach");
};

// Ring slot of output row offset x (compile-time after unrolling).
template <int P>
__device__ __forceinline__ constexpr int pslot(int x) { return ((x % P) + P) % P; }

// One CTA: a strip of 128 columns (64 column pairs, one per thread) of one instance and NS
// row streams of `srows` output rows each (stream st: rows a_lo[st] .. a_lo[st] + L[st] - 1,
// input rows from a_lo[st] - K), advanced in lockstep with a chunk ring each: independent
// instruction streams for the scheduler that share the T coefficients.  Input rows are
// processed in blocks of P (one turn of the accumulator rings, straight-line code).
template <int K, int NT, int NS>
__global__ void __launch_bounds__(Geo4<K, NT, NS>::NTH, Geo4<K, NT, NS>::MINB)
    k_apply_pcg4(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mQ,
                 const __grid_constant__ CUtensorMap mS, ApplyPcgArgs a, int srows) {
    using G = Geo4<K, NT, NS>;
    constexpr int P = G::P, SR = G::SR, KE = G::KE, CR = G::CR, D = G::D, RING = G::RING, NTH = G::NTH;
    constexpr unsigned DM = DiffMask<NT>::value;
    static_assert(DM & 1u, "term 0 is a difference term (exact mass split)");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    // rings of stream st: Z [RING][WCT], Q_prev [RING][WCT], coefficient rows [RING][SR]
    auto Zs = [&](int st) { return reinterpret_cast<float*>(sbase + (size_t)st * D * G::CHUNK_BYTES); };
    auto Qs = [&](int st) { return Zs(st) + RING * WCT; };
    auto Ss = [&](int st) { return Qs(st) + RING * WCT; };
    __shared__ __align__(8) unsigned long long bar[NS][D];
    __shared__ double red[NTH / 32];
    __shared__ float beta_s;
    __shared__ int fail_s, last_s;
    const int tid = threadIdx.x, inst = blockIdx.z;
    PcgScalars* sc = a.sc + inst;
    if (a.use_sc && !sc->active) return;
    const int b0 = blockIdx.x * TB;
    int a_lo[NS], L[NS], Lmax = 0;
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        a_lo[st] = (blockIdx.y * NS + st) * srows;
        L[st] = max(0, min(a.q, a_lo[st] + srows) - a_lo[st]);   // output rows of stream st
        Lmax = max(Lmax, L[st]);
    }
    const int nblk = (Lmax + 2 * K + P - 1) / P;                 // blocks of input rows
    const int nch = (nblk * P + CR - 1) / CR;                    // chunks per stream: input rows a_lo - K ...
    if (tid == 0) {
        for (int st = 0; st < NS; ++st)
            for (int i = 0; i < D; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[st][i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        beta_s = (a.use_sc && sc->iters > 0) ? (float)sc->beta : 0.f;
    }
    __syncthreads();
    // chunk c -> ring slot c % D: input rows a_lo - K + c CR .. of Z, Q_prev and the
    // coefficient table (rows outside [0, q) read as zeros)
    auto issue = [&](int st, int c) {
        const int slot = c % D;
        const uint32_t bb = smem_u32(&bar[st][slot]);
        const uint64_t pz = reinterpret_cast<uint64_t>(&mZ), pq = reinterpret_cast<uint64_t>(&mQ),
                       ps = reinterpret_cast<uint64_t>(&mS);
        const int x0 = b0 - XPAD, y0 = a_lo[st] - K + c * CR;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(G::CHUNK_BYTES)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Ss(st) + slot * G::SCH)), "l"(ps), "r"(bb), "r"(0), "r"(y0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Zs(st) + slot * G::ZCH)), "l"(pz), "r"(bb), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
            ::"r"(smem_u32(Qs(st) + slot * G::ZCH)), "l"(pq), "r"(bb), "r"(x0), "r"(y0), "r"(inst)
            : "memory");
    };
    if (tid == 0)
        for (int c = 0; c < D && c < nch; ++c)
            for (int st = 0; st < NS; ++st) issue(st, c);
    const int cp = tid;
    const int b = b0 + 2 * cp;
    const float* Tt = reinterpret_cast<const float*>(a.T);
    auto tload = [&](int il) -> float2 {
        const size_t o = (size_t)il * a.q + b;
        return make_float2(b < a.q ? Tt[o] : 0.f, b + 1 < a.q ? Tt[o + 1] : 0.f);
    };
    float2 tc[NT][P];
#pragma unroll
    for (int i = 0; i < NT; ++i)
#pragma unroll
        for (int l = 0; l < P; ++l) tc[i][l] = tload(i * P + l);
    // Term 0 exact mass split: X M_t^T = D (X + X N^T), N = D^{-1}(M_t - D) (zero row sums);
    // the s-pass acts on X and on X N^T separately, D scales the finished row.
    const float2 d0 = tc[0][K];
    {
        const float2 dinv = make_float2(d0.x != 0.f ? 1.f / d0.x : 0.f, d0.y != 0.f ? 1.f / d0.y : 0.f);
#pragma unroll
        for (int l = 0; l < P; ++l) tc[0][l] = (l == K) ? make_float2(0.f, 0.f) : f2mul(tc[0][l], dinv);
    }
    const float bsc = beta_s;
    const float2 beta2 = make_float2(bsc, bsc);
    float* Qn = reinterpret_cast<float*>(a.Qnew) + (size_t)inst * a.bs;
    float* LQ = reinterpret_cast<float*>(a.LQ) + (size_t)inst * a.bs;
    const bool col_ok = b < a.ld;   // pad columns [q, ld) receive zeros
    bool failed = false;
    int waited = 0, released = 0;
    auto wait_upto = [&](int need) {   // chunks 0 .. need-1 resident in every stream
        while (waited < need) {
#pragma unroll
            for (int st = 0; st < NS; ++st)
                if (!failed)
                    failed = !mbar_wait_bounded(smem_u32(&bar[st][waited % D]), (uint32_t)((waited / D) & 1));
            ++waited;
        }
    };
    const float2 zero2 = make_float2(0.f, 0.f);
    float2 acc0[NS][P], accR[NS][P], xr[NS][P];   // term-0 and other-term accumulators, new-direction centres
    float2 wprev[NS][NT];                         // previous input row's t-pass values (difference terms)
    float2 xprev[NS];
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        xprev[st] = zero2;
#pragma unroll
        for (int s = 0; s < P; ++s) {
            acc0[st][s] = zero2;
            accR[st][s] = zero2;
            xr[st][s] = zero2;
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) wprev[st][t] = zero2;
    }
    float2 dacc = zero2, zacc = zero2;   // <X, L(X)>, <Z, L(X)>
    // input index i (input row a_lo - K + i, staged at ring row i mod RING; u = i mod P):
    // t-pass, push into output rows i - 2K .. i (CTA-local), then output row i - 2K is done
    auto step = [&](const int st, int i, const int u) {
        const int rr = i & (RING - 1);
        const float2* z2 = reinterpret_cast<const float2*>(Zs(st) + rr * WCT + XPAD + 2 * cp - KE);
        const float2* q2 = reinterpret_cast<const float2*>(Qs(st) + rr * WCT + XPAD + 2 * cp - KE);
        float xs[2 * KE + 2];
#pragma unroll
        for (int m = 0; m <= KE; ++m) {
            const float2 v = f2fma(beta2, q2[m], z2[m]);
            xs[2 * m] = v.x;
            xs[2 * m + 1] = v.y;
        }
        const float2 xc = make_float2(xs[KE], xs[KE + 1]);
        {
            const int orow = i - K;   // the new direction's row of this centre
            if (orow >= 0 && orow < L[st] && col_ok)
                *reinterpret_cast<float2*>(Qn + (size_t)(a_lo[st] + orow) * a.ld + b) = xc;
        }
        float2 d[P];
#pragma unroll
        for (int l = 0; l < P; ++l)
            if (l != K) d[l] = f2sub(make_float2(xs[KE + l - K], xs[KE + l - K + 1]), xc);
        float2 w[NT];
        {
            float2 v = zero2;
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) v = f2fma(tc[0][l], d[l], v);
            w[0] = v;
        }
#pragma unroll
        for (int t = 1; t < NT; ++t) {
            float2 v = f2mul(tc[t][K], xc);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) v = f2fma(tc[t][l], d[l], v);
            w[t] = v;
        }
        // coefficients of this input row: term t at t P .. t P + 2K
        const float4* crow4 = reinterpret_cast<const float4*>(Ss(st) + rr * SR);
        auto cf = [&](int e) -> float2 {
            const float4 v = crow4[e >> 2];
            const float s = (e & 3) == 0 ? v.x : (e & 3) == 1 ? v.y : (e & 3) == 2 ? v.z : v.w;
            return make_float2(s, s);
        };
        {   // term 0, both parts of the split
            const float2 dx = f2sub(xc, xprev[st]), dw = f2sub(w[0], wprev[st][0]);
#pragma unroll
            for (int p = 0; p < 2 * K; ++p) {
                const float2 c = cf(p);
                const int s = pslot<P>(u - 2 * K + p);
                acc0[st][s] = f2fma(c, dx, acc0[st][s]);
                acc0[st][s] = f2fma(c, dw, acc0[st][s]);
            }
            const float2 c = cf(2 * K);
            const int s = pslot<P>(u - K);
            acc0[st][s] = f2fma(c, xc, acc0[st][s]);
            acc0[st][s] = f2fma(c, w[0], acc0[st][s]);
        }
#pragma unroll
        for (int t = 1; t < NT; ++t) {
            if ((DM >> t) & 1u) {
                const float2 dt = f2sub(w[t], wprev[st][t]);
#pragma unroll
                for (int p = 0; p < 2 * K; ++p) {
                    const int s = pslot<P>(u - 2 * K + p);
                    accR[st][s] = f2fma(cf(t * P + p), dt, accR[st][s]);
                }
                const int s = pslot<P>(u - K);
                accR[st][s] = f2fma(cf(t * P + 2 * K), w[t], accR[st][s]);
            } else {
#pragma unroll
                for (int p = 0; p <= 2 * K; ++p) {
                    const int s = pslot<P>(u - 2 * K + p);
                    accR[st][s] = f2fma(cf(t * P + p), w[t], accR[st][s]);
                }
            }
        }
        xprev[st] = xc;
#pragma unroll
        for (int t = 0; t < NT; ++t)
            if ((DM >> t) & 1u) wprev[st][t] = w[t];
        xr[st][pslot<P>(u - K)] = xc;
        {   // output row i - 2K: every input row that reaches it is in
            const int s = pslot<P>(u - 2 * K);
            const float2 y = f2fma(d0, acc0[st][s], accR[st][s]);
            const int jo = i - 2 * K;
            if (col_ok && jo >= 0 && jo < L[st]) {
                *reinterpret_cast<float2*>(LQ + (size_t)(a_lo[st] + jo) * a.ld + b) = y;
                dacc = f2fma(xr[st][s], y, dacc);
                const float2 zc =
                    *reinterpret_cast<const float2*>(Zs(st) + ((i - K) & (RING - 1)) * WCT + XPAD + 2 * cp);
                zacc = f2fma(zc, y, zacc);
            }
            acc0[st][s] = zero2;
            accR[st][s] = zero2;
        }
    };
#pragma unroll 1
    for (int m = 0; m < nblk; ++m) {
        const int i0 = m * P;
        const int iend = i0 + P;
        wait_upto(min(nch, (iend - 1) / CR + 1));
#pragma unroll
        for (int u = 0; u < P; ++u)
#pragma unroll
            for (int st = 0; st < NS; ++st) step(st, i0 + u, u);
        // chunks below the next block's oldest row (iend - K) are done: refill
        const int can = min(nch, (iend - K) / CR);
        if (can > released) {
            __syncthreads();   // every thread is past the rows of those slots
            if (tid == 0)
                for (int c = released; c < can; ++c)
                    if (c + D < nch)
                        for (int st = 0; st < NS; ++st) issue(st, c + D);
            released = can;
        }
    }
    wait_upto(nch);   // every issued copy has landed before the CTA exits
    if (failed) atomicOr(&fail_s, 1);
    const double sacc = block_sum<NTH>((double)dacc.x + (double)dacc.y, red);
    __syncthreads();   // red[] is reused
    const double s2v = a.partial2 ? block_sum<NTH>((double)zacc.x + (double)zacc.y, red) : 0.0;
    const int nb = gridDim.x * gridDim.y;
    if (tid == 0) {
        if (fail_s) atomicOr(a.status, DEV_ERR_TIMEOUT);
        a.partial[(size_t)inst * nb + blockIdx.y * gridDim.x + blockIdx.x] = sacc;
        if (a.partial2) a.partial2[(size_t)inst * nb + blockIdx.y * gridDim.x + blockIdx.x] = s2v;
        __threadfence();
        const unsigned t = atomicAdd(a.counter + inst, 1u);
        last_s = (t == (unsigned)nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (last_s && tid < 32) {
        __threadfence();
        const double qlq = warp_sum_partials(a.partial + (size_t)inst * nb, nb);
        const double lqz = a.partial2 ? warp_sum_partials(a.partial2 + (size_t)inst * nb, nb) : 0.0;
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

// Resident CTAs of the push-form apply on the current device (one wave).
template <int K, int NT, int NS>
int apply4_ctas_wanted_t() {
    using G = Geo4<K, NT, NS>;
    static std::atomic<int> cache[MOFEM_MAX_DEV];
    const int slot = dev_slot();
    int n = cache[slot].load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
        smem_attr_once(k_apply_pcg4<K, NT, NS>, (int)G::SMEM, attr_done);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_pcg4<K, NT, NS>, G::NTH, G::SMEM) !=
                cudaSuccess ||
            per < 1)
            per = 1;
        n = (sms > 0 ? sms : 1) * per;
        cache[slot].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Output rows per segment: the segment and its 2K halo rows fill whole blocks of P input
// rows (only the last segment is ragged).
inline int apply4_rows(int q, int segs, int K, int ns) {
    const int P = 2 * K + 1;
    const int per = (q + segs * ns - 1) / (segs * ns);
    return (per + 2 * K + P - 1) / P * P - 2 * K;
}

// Row streams per thread of the push-form apply.
__host__ __device__ constexpr int push_streams(int, int) { return 1; }

template <int K, int NT>
mofem_status launch_pcg4_t(const CUtensorMap& mZ, const CUtensorMap& mQ, const CUtensorMap& mS,
                           const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    constexpr int NS = push_streams(K, NT);
    using G = Geo4<K, NT, NS>;
    auto kern = k_apply_pcg4<K, NT, NS>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)G::SMEM, attr_done));
    const int strips = (a.q + TB - 1) / TB;
    const int segs = apply3_segments(a.q, strips, batch, apply4_ctas_wanted_t<K, NT, NS>() * max(1, a.seg_div), K, NS);
    const int srows = apply4_rows(a.q, segs, K, NS);
    dim3 grid(strips, segs, batch);
    kern<<<grid, G::NTH, G::SMEM, st>>>(mZ, mQ, mS, a, srows);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
