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
//     (the NT (2K + 1) coefficients of a row contiguous, the row padded to a
//     multiple of 8 floats); a shared-memory read delivers 128 bytes per
//     wavefront whether or not the lanes share the address, so each lane reads
//     every coefficient once and pairs it in registers for the paired FMAs.
//
// Fused epilogue: per-CTA FP64 partials of <X, L(X)> and <L(X), Z> and, in the
// last CTA of each instance, alpha = <R, Z> / <Q, L(Q)> and the flexible-beta
// numerator term <R_new, Z> = <R, Z> - alpha <L(Q), Z> (fixed-order sums of the
// partials), so the residual update never reads Z again.
#pragma once
#include "apply_impl.cuh"

namespace mofem_apply_impl {

template <int K, int NT, int NS>
struct Geo3 {
    static constexpr int P = 2 * K + 1;
    static constexpr int NTH = 64;                       // threads = column pairs per CTA
    static constexpr int CR = 4;                         // rows per staged chunk
    static constexpr int D = 4;                          // chunks in each stream's ring
    static constexpr int RING = CR * D;                  // staged rows per stream (power of two)
    static constexpr int RELEASE = 1;                    // chunks released (and refilled) together
    // register-ring slots of t-pass rows: one more than the stencil needs (2K + 1), so that
    // the t-pass of the next row writes a slot the current row's s-pass does not read and
    // the two can overlap; rows are unrolled by RSLOT.  Where the chunk ring is too short
    // for the longer block, the stencil's own 2K + 1.
    static constexpr int RSLOT = (D - RELEASE) * CR >= 4 * K + 1 ? P + 1 : P;
    static constexpr int SR = ((NT * P + 7) / 8) * 8;    // floats per S row (a chunk of CR = 4 S rows
                                                         // stays a 128-byte multiple)
    static constexpr bool TREG = NT * P <= 25;           // T coefficients in registers, else shared
    static constexpr int KE = K + (K & 1);               // left reach rounded to an even column
    static constexpr int ZCH = CR * WCT;                 // floats per chunk of Z (and of Q_prev)
    static constexpr int SCH = CR * SR;                  // floats per chunk of S rows
    static constexpr uint32_t CHUNK_BYTES = 2u * ZCH * 4u + (uint32_t)SCH * 4u;
    static constexpr uint32_t STREAM_BYTES = (uint32_t)D * CHUNK_BYTES;
    static constexpr size_t SMEM = (size_t)NS * STREAM_BYTES + (TREG ? 0 : (size_t)NT * P * NTH * 8) + 128;
    // register budget: the T coefficients (in registers when TREG) serve every stream of
    // the thread; one stream with the extra slot fits 204 registers (5 resident CTAs), two
    // streams 255 (4 CTAs)
    static constexpr int MINB = NS == 1 ? (TREG ? 5 : 4) : 4;
    static_assert((RING & (RING - 1)) == 0, "ring rows must be a power of two");
    static_assert((ZCH * 4) % 128 == 0 && (SCH * 4) % 128 == 0, "TMA destinations stay 128-byte aligned");
    // a chunk is refilled only after its last row is done, RELEASE chunks at a time; the rows
    // that wait for it must not be the ones that release it:
    // (D - RELEASE) CR >= 2K (t-pass reach) + RSLOT - 1 (unrolled block)
    static_assert((D - RELEASE) * CR >= 2 * K + RSLOT - 1, "ring too short for the stencil reach");
    static_assert(NS == 1 || TREG, "two streams per thread only with the T coefficients in registers");
};

// Operator forms served by the packed kernel (the ring and, if TREG, the T
// coefficients live in registers); the others use k_apply_pcg.
__host__ __device__ constexpr bool packed_apply_ok(int K, int NT) { return NT * (2 * K + 1) <= 40; }
// Row streams per thread of the packed kernel.  Two streams share the T coefficients and
// cut the instructions by 17% (P2 2049 x 4), but at 255 registers only 8 warps fit per SM
// and the launch took 100.8 us against 98.6 for one stream: the shared-memory pipe (66% of
// peak in both) is what the two forms share; one stream is kept.
__host__ __device__ constexpr int packed_streams(int, int) { return 1; }

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - c, one rounding (fma with an exact -1 product)
__device__ __forceinline__ float2 f2sub(float2 a, float2 c) { return __ffma2_rn(c, make_float2(-1.f, -1.f), a); }

// Number of segments per strip: at most one wave of resident CTAs over all strips and
// instances (a partial second wave would double the time of the SMs that run it), at
// least 8 (2K + 8) rows per stream.
__host__ __device__ inline int apply3_segments(int q, int strips, int batch, int ctas_wanted, int K, int ns) {
    const int min_rows = 8 * (2 * K + 8) * ns;
    int segs = ctas_wanted / (strips * batch);
    const int max_segs = (q + min_rows - 1) / min_rows;
    if (segs > max_segs) segs = max_segs;
    return segs < 1 ? 1 : segs;
}

// One CTA: a strip of 128 columns (64 column pairs, one per thread) of one instance and a
// segment of rows, split into NS row streams of `srows` rows that the thread advances in
// lockstep (independent instruction streams for the scheduler; the T coefficients are
// loaded once and serve all of them).  Each stream has its own TMA chunk ring.
template <int K, int NT, int NS>
__global__ void __launch_bounds__(Geo3<K, NT, NS>::NTH, Geo3<K, NT, NS>::MINB)
    k_apply_pcg3(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mQ,
                 const __grid_constant__ CUtensorMap mS, ApplyPcgArgs a, int srows) {
    using G = Geo3<K, NT, NS>;
    constexpr int P = G::P, SR = G::SR, KE = G::KE, CR = G::CR, D = G::D, RING = G::RING, NTH = G::NTH;
    constexpr unsigned DM = DiffMask<NT>::value;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    // stream s: Z ring [RING][WCT], Q_prev ring [RING][WCT], S ring [RING][SR]
    auto Zs = [&](int st) { return reinterpret_cast<float*>(sbase + st * G::STREAM_BYTES); };
    auto Qs = [&](int st) { return Zs(st) + RING * WCT; };
    auto Ss = [&](int st) { return Qs(st) + RING * WCT; };
    float2* T2s = reinterpret_cast<float2*>(sbase + NS * G::STREAM_BYTES);   // [NT*P][NTH] (!TREG)
    __shared__ __align__(8) unsigned long long bar[NS][D];
    __shared__ double red[NTH / 32];
    __shared__ float beta_s;
    __shared__ int fail_s, last_s;
    const int tid = threadIdx.x, inst = blockIdx.z;
    PcgScalars* sc = a.sc + inst;
    if (a.use_sc && !sc->active) return;
    const int b0 = blockIdx.x * TB;
    int a_lo[NS], L[NS];
    int Lmax = 0;
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        a_lo[st] = (blockIdx.y * NS + st) * srows;
        L[st] = max(0, min(a.q, a_lo[st] + srows) - a_lo[st]);   // output rows of stream st
        Lmax = max(Lmax, L[st]);
    }
    // rows are computed in whole blocks of RSLOT (straight-line code, stores guarded): a
    // block may run past L into zero-filled or neighbouring rows, never stored
    constexpr int RS = G::RSLOT;
    const int nblk_rows = (Lmax + RS - 1) / RS;
    const int nch = (nblk_rows * RS + 2 * K + CR - 1) / CR;   // chunks of each stream: input rows a_lo - K ...
    if (tid == 0) {
        for (int st = 0; st < NS; ++st)
            for (int i = 0; i < D; ++i)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[st][i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
        beta_s = (a.use_sc && sc->iters > 0) ? (float)sc->beta : 0.f;
    }
    __syncthreads();
    // chunk c of stream st -> its ring slot c % D: input rows a_lo - K + c CR .. (Z, Q_prev)
    // and S rows a_lo + c CR ..
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
            ::"r"(smem_u32(Ss(st) + slot * G::SCH)), "l"(ps), "r"(bb), "r"(0), "r"(a_lo[st] + c * CR), "r"(inst)
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
    int waited = 0, released = 0;   // chunks, the same count in every stream (lockstep)
    auto wait_upto = [&](int need) {   // chunks 0 .. need-1 resident in every stream
        while (waited < need) {
#pragma unroll
            for (int st = 0; st < NS; ++st)
                if (!failed)
                    failed = !mbar_wait_bounded(smem_u32(&bar[st][waited % D]), (uint32_t)((waited / D) & 1));
            ++waited;
        }
    };
    float2 ring[NS][NT][RS];
    float2 xr0[NS][RS];
    // t-pass of input index i (input row a_lo - K + i, staged at ring row ri) of stream st
    // into register-ring slot `slot`
    auto tpass = [&](int st, int i, int ri, int slot) {
        const int rr = ri * WCT + XPAD + 2 * cp - KE;
        const float2* z2 = reinterpret_cast<const float2*>(Zs(st) + rr);
        const float2* q2 = reinterpret_cast<const float2*>(Qs(st) + rr);
        float xs[2 * KE + 2];
#pragma unroll
        for (int m = 0; m <= KE; ++m) {
            const float2 v = f2fma(beta2, q2[m], z2[m]);
            xs[2 * m] = v.x;
            xs[2 * m + 1] = v.y;
        }
        const float2 xc = make_float2(xs[KE], xs[KE + 1]);
        xr0[st][slot] = xc;
        const int orow = i - K;   // stream output row whose centre this is
        if (orow >= 0 && orow < L[st] && col_ok)
            *reinterpret_cast<float2*>(Qn + (size_t)(a_lo[st] + orow) * a.ld + b) = xc;
        float2 d[P];
#pragma unroll
        for (int l = 0; l < P; ++l)
            if (l != K) d[l] = f2sub(make_float2(xs[KE + l - K], xs[KE + l - K + 1]), xc);
        {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = f2fma(n0[l], d[l], w);
            ring[st][0][slot] = w;
        }
#pragma unroll
        for (int t = 1; t < NT; ++t) {
            float2 w = f2mul(tcoef(t, K), xc);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l != K) w = f2fma(tcoef(t, l), d[l], w);
            ring[st][t][slot] = w;
        }
    };
    float2 acc = make_float2(0.f, 0.f), acz = make_float2(0.f, 0.f);
    // s-pass of stream output row j (register-ring slots of input rows j .. j + 2K at
    // (u + jj) % RSLOT; its S row staged at ring row rs, the Z centre at ring row rc)
    auto spass = [&](int st, int j, int u, int rs, int rc) {
        const float4* srow4 = reinterpret_cast<const float4*>(Ss(st) + rs * SR);
        auto sc2 = [&](int e) -> float2 {   // coefficient e in both lanes (float4 e/4 holds e .. e+3)
            const float4 v = srow4[e >> 2];
            const float s = (e & 3) == 0 ? v.x : (e & 3) == 1 ? v.y : (e & 3) == 2 ? v.z : v.w;
            return make_float2(s, s);
        };
        float2 yt[NT];
        {
            const float2 xc = xr0[st][(u + K) % RS], wc = ring[st][0][(u + K) % RS];
            float2 ya = f2mul(sc2(K), xc), yb = f2mul(sc2(K), wc);
#pragma unroll
            for (int jj = 0; jj < P; ++jj)
                if (jj != K) {
                    ya = f2fma(sc2(jj), f2sub(xr0[st][(u + jj) % RS], xc), ya);
                    yb = f2fma(sc2(jj), f2sub(ring[st][0][(u + jj) % RS], wc), yb);
                }
            yt[0] = f2mul(d0, f2add(ya, yb));
        }
#pragma unroll
        for (int t = 1; t < NT; ++t) {
            const float2 wc = ring[st][t][(u + K) % RS];
            float2 y = f2mul(sc2(t * P + K), wc);
#pragma unroll
            for (int jj = 0; jj < P; ++jj)
                if (jj != K) {
                    if ((DM >> t) & 1u) y = f2fma(sc2(t * P + jj), f2sub(ring[st][t][(u + jj) % RS], wc), y);
                    else y = f2fma(sc2(t * P + jj), ring[st][t][(u + jj) % RS], y);
                }
            yt[t] = y;
        }
        // pairwise sum of the term results (independent chains above)
#pragma unroll
        for (int s2 = 1; s2 < NT; s2 *= 2)
#pragma unroll
            for (int t = 0; t + s2 < NT; t += 2 * s2) yt[t] = f2add(yt[t], yt[t + s2]);
        const float2 y = yt[0];
        if (col_ok && j < L[st]) {
            *reinterpret_cast<float2*>(LQ + (size_t)(a_lo[st] + j) * a.ld + b) = y;
            acc = f2fma(xr0[st][(u + K) % RS], y, acc);
            const float2 zc = *reinterpret_cast<const float2*>(Zs(st) + rc * WCT + XPAD + 2 * cp);
            acz = f2fma(zc, y, acz);
        }
    };
    wait_upto(min(nch, (2 * K - 1) / CR + 1));
#pragma unroll
    for (int r = 0; r < 2 * K; ++r)
#pragma unroll
        for (int st = 0; st < NS; ++st) tpass(st, r, r, r);
#pragma unroll 1
    for (int m = 0; m < nblk_rows; ++m) {
        const int j0 = m * RS;
        const int jend = j0 + RS;
        wait_upto(min(nch, (jend - 1 + 2 * K) / CR + 1));
#pragma unroll
        for (int u = 0; u < RS; ++u) {
            const int j = j0 + u;   // stream output row
            // staged ring rows of the t-pass input (j + 2K), the S row (j), the Z centre (j + K)
            const int zr = (j + 2 * K) & (RING - 1), sr = j & (RING - 1), cr = (j + K) & (RING - 1);
#pragma unroll
            for (int st = 0; st < NS; ++st) tpass(st, j + 2 * K, zr, (u + 2 * K) % RS);
#pragma unroll
            for (int st = 0; st < NS; ++st) spass(st, j, u, sr, cr);
        }
        // chunks whose last row (its S rows end at output row (c + 1) CR - 1) is done: refill,
        // RELEASE chunks at a time (fewer barriers)
        int can = min(nch, jend / CR);
        if (can < nch) can -= (can - released) % G::RELEASE;
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
    double sacc = block_sum<NTH>((double)acc.x + (double)acc.y, red);
    __syncthreads();   // red[] is reused
    const double s2v = a.partial2 ? block_sum<NTH>((double)acz.x + (double)acz.y, red) : 0.0;
    const int nblk = gridDim.x * gridDim.y;
    if (tid == 0) {
        if (fail_s) atomicOr(a.status, DEV_ERR_TIMEOUT);
        a.partial[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = sacc;
        if (a.partial2) a.partial2[(size_t)inst * nblk + blockIdx.y * gridDim.x + blockIdx.x] = s2v;
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

// Resident CTAs of the streaming apply on the current device (one wave), per form.
template <int K, int NT, int NS>
int apply3_ctas_wanted_t() {
    using G = Geo3<K, NT, NS>;
    static std::atomic<int> cache[MOFEM_MAX_DEV];
    const int slot = dev_slot();
    int n = cache[slot].load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
        smem_attr_once(k_apply_pcg3<K, NT, NS>, (int)G::SMEM, attr_done);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_apply_pcg3<K, NT, NS>, G::NTH, G::SMEM) !=
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
    constexpr int NS = packed_streams(K, NT);
    using G = Geo3<K, NT, NS>;
    auto kern = k_apply_pcg3<K, NT, NS>;
    static std::atomic<bool> attr_done[MOFEM_MAX_DEV];
    MOFEM_CUDA_TRY(smem_attr_once(kern, (int)G::SMEM, attr_done));
    const int strips = (a.q + TB - 1) / TB;
    const int segs = apply3_segments(a.q, strips, batch, apply3_ctas_wanted_t<K, NT, NS>() * max(1, a.seg_div), K, NS);
    constexpr int P = 2 * K + 1;   // streams of whole row blocks: only the last one is ragged
    const int srows = ((a.q + segs * NS - 1) / (segs * NS) + P - 1) / P * P;
    dim3 grid(strips, segs, batch);
    kern<<<grid, G::NTH, G::SMEM, st>>>(mZ, mQ, mS, a, srows);
    MOFEM_CUDA_TRY(cudaGetLastError());
    return MOFEM_OK;
}

}  // namespace mofem_apply_impl
