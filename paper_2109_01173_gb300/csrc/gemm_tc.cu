// tcgen05 tensor-core GEMMs of the reduced-approach preconditioner
// (Sec. 4, Eq. reduced_formula_for_u, applied to the two-term Sylvester
// preconditioner of MO-PCG):
//
//     Z = Q1 ((Q1^T R Q2) ./ (lambda_a + mu_b)) Q2^T
//
// computed as four GEMMs, each of the form D = A B^T with both operands
// "K-major" (row-major, contraction index contiguous), the output D stored in
// its natural row-major layout, which is exactly the K-major operand the next
// GEMM needs:
//   G1: D[j][a] = sum_b Q2T[j][b] R[a][b]     -> X1T[j][a]   (X1 = R Q2)
//   G2: D[j][i] = sum_a X1T[j][a] Q1T[i][a]   -> WT[j][i] = D / (lam_i + mu_j)
//   G3: D[a][j] = sum_i Q1[a][i] WT[j][i]     -> Y[a][j]     (Y = Q1 W)
//   G4: D[a][b] = sum_j Y[a][j] Q2[b][j]      -> Z[a][b]     (Z = Y Q2^T), + <R, Z> partials
//
// Kernel (k_gemm_2sm): a persistent grid of CTA pairs (2-CTA clusters, one CTA
// per SM) walking all 256 x 256 output tiles of all instances.  Each pair
// computes one tile with tcgen05.mma.cta_group::2 (M = 256 split over the two
// SMs' TMEM lanes, N = 256 FP32 TMEM columns): CTA r stages rows 128 r .. of the
// A and of the B slice of every 128-byte K step (SWIZZLE_128B TMA boxes, 6-stage
// ring of 32 KB), the leader CTA issues the MMAs (kind::f16 with FP16/BF16
// operands, or kind::tf32), and two TMEM accumulators let the epilogue
// (tcgen05.ld 32x32b.x32) of one tile overlap the mainloop of the next.  Every
// mbarrier wait is bounded (2 s of %globaltimer); on expiry the CTA records
// DEV_ERR_TIMEOUT, stops all roles, frees its TMEM and exits (the peer then
// times out as well).
#include "internal.h"

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdio>

namespace {

constexpr int BM = 128, BN = 256;   // output rows per CTA (TMEM lanes), columns per tile
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

enum { EPI_STORE = 0, EPI_DIV = 1, EPI_Z = 2 };

struct GemmArgs {
    void* out; long long out_bs; int out_ld; int out_bf16;   // out_bf16: 0 FP32, 1 BF16, 2 FP16 output
    int M, N, nk, batch;
    int a_shared, b_shared;
    int epi;
    const float* lam; long long lam_bs; const float* mu;
    const float* R; long long r_bs; int r_ld;
    double* rz_part;
    PcgScalars* sc;       // skip inactive instances; with rz_part, last-CTA beta finalisation
    unsigned* counter;    // [batch] CTA tickets (zeroed, self-resetting)
    int flex;
    int div_product;       // EPI_DIV divisor lambda_i * mu_j (product preconditioner) instead of lambda_i + mu_j
    const PcgScalars* scl; // FP16 operands: the G4 output is divided by scl[inst].rscale
    int* status;
    int pad_ok;            // the output's row padding (columns N .. round_up(N, 32) - 1 <= out_ld) may be
                           // written with zeros: the ragged last chunk then takes 16-byte stores
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with cluster-scope acquire: for data the partner CTA stored into this CTA's
// shared memory before its release arrive
__device__ __forceinline__ bool mbar_try_cl(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, "
        "0, p;\n}\n"
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
// Shared-memory matrix descriptor: K-major tile written by TMA with 128-byte
// swizzle (8-row x 128-byte atoms, 1024 bytes apart), tcgen05 descriptor version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Shared pieces of the persistent, warp-specialised GEMM: 192 threads,
//   warps 0-3 : epilogue (TMEM lanes 0-127 = output rows), overlapping the next
//               tile's mainloop thanks to two TMEM accumulators (2 x 256 columns)
//   warp 4    : TMA producer
//   warp 5    : TMEM allocation and tcgen05.mma issue (one elected lane)
// Every wait is bounded; a timeout raises a CTA-wide abort flag that ends all roles.
constexpr int P_THREADS = 192;
constexpr uint32_t TMEM_COLS_P = 512;

__device__ __forceinline__ bool pwait(uint32_t a, uint32_t parity, volatile int* abort) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(a, parity)) {
        if (*abort) return false;
        if (gtimer() - t0 > WAIT_LIMIT_NS) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// Epilogue of one 32-column chunk held by this thread (row m): divide (G2), unscale
// and <R, Z> accumulation (G4), store (16-byte vectors when aligned).  Specialised
// at compile time on the epilogue kind and the output type (OUTK 0 FP32, 1 BF16,
// 2 FP16): one small code path per GEMM (a generic epilogue with every path inlined
// cost 10-20% of the GEMM's time).
template <int EPI, int OUTK>
__device__ __forceinline__ void epi_chunk(const GemmArgs& g, int inst, int m, int nb, float (&v)[32], float mu_m,
                                          float inv_scale, double& acc) {
    const size_t obase = (size_t)inst * g.out_bs + (size_t)m * g.out_ld;
    if constexpr (EPI == EPI_DIV) {
        // lambda of the chunk's 32 columns: 16-byte read-only loads (the rows of lam are
        // ld-strided, ld a multiple of 64, and nb a multiple of 32: 128-byte aligned)
        const float4* lam4 = reinterpret_cast<const float4*>(g.lam + (size_t)inst * g.lam_bs + nb);
        float lam[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 t = __ldg(lam4 + j);
            lam[4 * j] = t.x; lam[4 * j + 1] = t.y; lam[4 * j + 2] = t.z; lam[4 * j + 3] = t.w;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __fdividef(v[j], g.div_product ? lam[j] * mu_m : lam[j] + mu_m);
    }
    if constexpr (EPI == EPI_Z) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= inv_scale;
    }
    // ragged last chunk: zero the columns >= N and store whole vectors where the padding
    // may be written (scalar sub-word stores into one sector serialise: 10-15% of a GEMM)
    const bool fits = nb + 32 <= g.N;
    const bool padw = !fits && g.pad_ok && nb + 32 <= g.out_ld;
    if (padw) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (nb + j >= g.N) v[j] = 0.f;
    }
    if constexpr (OUTK != 0) {
        const bool full = (g.out_ld % 8) == 0 && (fits || padw);
        if constexpr (OUTK == 2) {   // FP16 intermediates: saturate instead of overflowing to inf
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fminf(fmaxf(v[j], -65504.f), 65504.f);
        }
        using OT = typename std::conditional<OUTK == 2, __half, __nv_bfloat16>::type;
        OT* o = reinterpret_cast<OT*>(g.out) + obase + nb;
        if (full) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if constexpr (OUTK == 2) {
                        __half2 t = __floats2half2_rn(v[j + 2 * e], v[j + 2 * e + 1]);
                        w[e] = *reinterpret_cast<uint32_t*>(&t);
                    } else {
                        __nv_bfloat162 t = __floats2bfloat162_rn(v[j + 2 * e], v[j + 2 * e + 1]);
                        w[e] = *reinterpret_cast<uint32_t*>(&t);
                    }
                }
                *reinterpret_cast<uint4*>(o + j) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else {
            for (int j = 0; j < 32 && nb + j < g.N; ++j) {
                if constexpr (OUTK == 2) o[j] = __float2half_rn(v[j]);
                else o[j] = __float2bfloat16_rn(v[j]);
            }
        }
    } else {
        float* o = reinterpret_cast<float*>(g.out) + obase + nb;
        const float* r = (EPI == EPI_Z && g.R) ? g.R + (size_t)inst * g.r_bs + (size_t)m * g.r_ld + nb : nullptr;
        float a32 = 0.f;   // FP32 within the 32-column chunk, FP64 across chunks
        const bool full = (g.out_ld % 4) == 0 && (fits || (padw && (!r || nb + 32 <= g.r_ld)));
        if (full && (!r || (g.r_ld % 4) == 0)) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                if (EPI == EPI_Z && r) {
                    float4 rv = *reinterpret_cast<const float4*>(r + j);
                    if (!fits) {   // padding of R contributes nothing, whatever it holds
                        if (nb + j >= g.N) rv.x = 0.f;
                        if (nb + j + 1 >= g.N) rv.y = 0.f;
                        if (nb + j + 2 >= g.N) rv.z = 0.f;
                        if (nb + j + 3 >= g.N) rv.w = 0.f;
                    }
                    a32 = fmaf(v[j], rv.x, a32);
                    a32 = fmaf(v[j + 1], rv.y, a32);
                    a32 = fmaf(v[j + 2], rv.z, a32);
                    a32 = fmaf(v[j + 3], rv.w, a32);
                }
            }
        } else {
            for (int j = 0; j < 32 && nb + j < g.N; ++j) {
                o[j] = v[j];
                if (EPI == EPI_Z && r) a32 = fmaf(v[j], r[j], a32);
            }
        }
        if constexpr (EPI == EPI_Z) acc += (double)a32;
    }
}

// ---------------------------------------------------------------------------
// TMA-store epilogue.  Each epilogue warp owns 32 output rows of the CTA's 128; it stages
// one block of 128-byte rows (32 FP32 or 64 16-bit columns) in a shared-memory buffer
// whose 16-byte chunks are XOR-swizzled by (row & 7) (the SWIZZLE_128B layout of the
// store's tensor map, so the writes of 8 consecutive rows hit all 32 banks), and one lane
// stores the block with cp.async.bulk.tensor: full 128-byte lines instead of 32 scattered
// 16-byte row pieces per warp store; the map clips rows and columns past the matrix.  Two
// buffers per warp alternate; a buffer is rewritten only after the store issued from it
// two blocks earlier has read it.
constexpr int EPI_STAGE_BYTES = 4096;   // 32 rows x 128 bytes per warp and buffer
constexpr int EPI_STAGE_TOTAL = 4 * 2 * EPI_STAGE_BYTES;

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Epilogue arithmetic of one 32-column chunk of row m (no store): divide (G2), unscale
// and <R, Z> accumulation (G4).  Same operations and order as epi_chunk.
template <int EPI>
__device__ __forceinline__ void epi_math(const GemmArgs& g, int inst, int m, int nb, float (&v)[32], float mu_m,
                                         float inv_scale, double& acc) {
    if constexpr (EPI == EPI_DIV) {
        const float4* lam4 = reinterpret_cast<const float4*>(g.lam + (size_t)inst * g.lam_bs + nb);
        float lam[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 t = __ldg(lam4 + j);
            lam[4 * j] = t.x; lam[4 * j + 1] = t.y; lam[4 * j + 2] = t.z; lam[4 * j + 3] = t.w;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __fdividef(v[j], g.div_product ? lam[j] * mu_m : lam[j] + mu_m);
    }
    if constexpr (EPI == EPI_Z) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] *= inv_scale;
        if (g.R) {
            const float* r = g.R + (size_t)inst * g.r_bs + (size_t)m * g.r_ld + nb;
            float a32 = 0.f;   // FP32 within the 32-column chunk, FP64 across chunks
            if (nb + 32 <= g.N && (g.r_ld % 4) == 0) {
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const float4 rv = *reinterpret_cast<const float4*>(r + j);
                    a32 = fmaf(v[j], rv.x, a32);
                    a32 = fmaf(v[j + 1], rv.y, a32);
                    a32 = fmaf(v[j + 2], rv.z, a32);
                    a32 = fmaf(v[j + 3], rv.w, a32);
                }
            } else {
                for (int j = 0; j < 32 && nb + j < g.N; ++j) a32 = fmaf(v[j], r[j], a32);
            }
            acc += (double)a32;
        }
    }
}

// Row `lane` of a staged block: the half-th 32-column chunk of it (half = 0 for FP32
// blocks, 0 or 1 for 16-bit ones), 16-byte pieces swizzled by (lane & 7).
template <int OUTK>
__device__ __forceinline__ void stage_chunk(uint8_t* buf, int lane, int half, const float (&v)[32]) {
    uint4* row = reinterpret_cast<uint4*>(buf + lane * 128);
    const int sw = lane & 7;
    if constexpr (OUTK == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            row[k ^ sw] = make_uint4(__float_as_uint(v[4 * k]), __float_as_uint(v[4 * k + 1]),
                                     __float_as_uint(v[4 * k + 2]), __float_as_uint(v[4 * k + 3]));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float a = v[8 * k + 2 * e], b = v[8 * k + 2 * e + 1];
                if constexpr (OUTK == 2) {   // FP16 intermediates: saturate instead of overflowing to inf
                    a = fminf(fmaxf(a, -65504.f), 65504.f);
                    b = fminf(fmaxf(b, -65504.f), 65504.f);
                    __half2 t = __floats2half2_rn(a, b);
                    w[e] = *reinterpret_cast<uint32_t*>(&t);
                } else {
                    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
                    w[e] = *reinterpret_cast<uint32_t*>(&t);
                }
            }
            row[(half * 4 + k) ^ sw] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// The whole 256-column tile row block of this warp through the staging buffers.
template <int EPI, int OUTK>
__device__ __forceinline__ void epi_tile_tma(const GemmArgs& g, const CUtensorMap* omap, uint32_t tm, int inst,
                                             int m, bool m_ok, int m_warp0, int n0, float mu_m, float inv_scale,
                                             double& acc, uint8_t* stage, int warp, int lane, int& nst) {
    constexpr int W = OUTK == 0 ? 32 : 64;   // columns per 128-byte staged row
#pragma unroll 1
    for (int blk = 0; blk < 256 / W; ++blk) {
        if (nst >= 2) {   // the store issued from this buffer two blocks ago has read it
            if (lane == 0) bulk_wait_read1();
            __syncwarp();
        }
        uint8_t* buf = stage + (warp * 2 + (nst & 1)) * EPI_STAGE_BYTES;
#pragma unroll
        for (int h = 0; h < W / 32; ++h) {
            const int c = blk * (W / 32) + h;
            float v[32];
            tmem_ld32(tm + (uint32_t)(c * 32), v);
            const int nb = n0 + c * 32;
            if (m_ok && nb < g.N) epi_math<EPI>(g, inst, m, nb, v, mu_m, inv_scale, acc);
            stage_chunk<OUTK>(buf, lane, h, v);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            tma_store_3d(omap, smem_u32(buf), n0 + blk * W, m_warp0, inst);
            bulk_commit();
        }
        ++nst;
    }
}

// ---------------------------------------------------------------------------
// k_gemm_2sm: each 2-CTA cluster computes one 256 x 256 tile with
// tcgen05.mma.cta_group::2 (M = 256 across the pair, N = 256).  CTA r holds rows
// 128 r .. 128 r + 127 of the A slice and of the B slice of every K step in its
// own shared memory (32 KB per stage, 6 stages); the leader CTA (rank 0) issues
// the MMAs, which read both CTAs' halves and write D rows 128 r .. 128 r + 127
// (all 256 columns) into CTA r's TMEM.  Both CTAs' TMA loads complete on the
// leader's stage barrier; the leader's commits release the stage and the
// finished accumulator in both CTAs (multicast); both CTAs' epilogue warps
// release an accumulator on the leader's barrier.  Each SM receives 32 KB per
// 512 tensor cycles instead of 48 KB (the K-slice bytes per MMA are what bound
// the 1-SM tiles).
#ifndef MOFEM_GEMM_STAGES
#define MOFEM_GEMM_STAGES 6   // 32 KB stages in flight per CTA
#endif
constexpr int ST2 = MOFEM_GEMM_STAGES;
constexpr int A2_BYTES = 128 * 128, B2_BYTES = 128 * 128;
constexpr int STAGE2_BYTES = A2_BYTES + B2_BYTES;

constexpr int NU = 8;   // unit ring of a chain launch: tile indices taken, not yet consumed by every role
struct PBars2 {
    uint64_t full[ST2], empty[ST2], tfull[2], tempty[2];
    uint64_t ufull[NU], uempty[NU];
    int uslot[NU];
    uint32_t tmem_slot;
    int abort;
    int mode;   // chain tile order of this launch (1 static, 2 dynamic)
    double red[2][4];
};

__device__ __forceinline__ uint32_t mapa_shared(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, uint32_t mbar_cluster, int c0,
                                                 int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar_cluster), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__host__ __device__ constexpr uint32_t make_idesc2(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}
template <int KIND>
__device__ __forceinline__ void mma2(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(make_idesc2(2)), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d), "l"(a), "l"(b), "r"(make_idesc2(KIND == 2 ? 0u : 1u)), "r"(acc)
            : "memory");
    }
}
__device__ __forceinline__ void commit2_mc(uint32_t mbar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
        ::"r"(mbar), "h"(mask)
        : "memory");
}

// A chain of GEMMs in one persistent launch (the preconditioner's G1..G4): the
// pairs walk the tiles of all stages in stage-major order; a tile of stage s > 0
// whose operand is stage s-1's output waits (bounded) until the 256-row output panel
// it reads is complete, counted by the four epilogue warps of both CTAs of every
// tile of that panel.  Two tile orders:
//  - static round-robin (pair p: tiles p, p + P, ...): the fastest (0.7 ms per
//    P2 2049 x 4 solve ahead of the dynamic order), but a pair may wait on a tile of
//    a pair that is not resident yet, so it is taken only by a launch that is alone
//    among chain launches on the device (g_chain_inflight);
//  - dynamic: each pair's leader takes the next tile from a global counter, so a
//    tile waits only on smaller indices taken earlier by running pairs and the
//    smallest unfinished tile can always proceed, however many pairs are resident.
// One launch instead of four saves three launch / prologue / pipeline-fill /
// last-epilogue latencies (~9.5 us each at P2 2049 x 4), and the next stage's tiles
// fill the previous one's tail.
constexpr int CHAIN_MAX = 4;
struct GemmChain {
    CUtensorMap mA[CHAIN_MAX], mB[CHAIN_MAX];
    CUtensorMap mO[CHAIN_MAX];   // output maps of the TMA-store epilogue (128-byte swizzled rows)
    int ostore[CHAIN_MAX];       // 1: the stage's output leaves through shared memory by TMA stores
    GemmArgs g[CHAIN_MAX];   // per stage; M, N, nk, batch, sc and status are the same in all
    int dep[CHAIN_MAX];      // operand from stage s-1: 0 none, 1 the A rows (panel = tile row),
                             // 2 the B rows (panel = tile column)
    int ns;                  // stages in this launch
    unsigned* panel_cnt;     // [stage][batch][row panel]: finished CTA tiles (null: ns == 1)
    unsigned* end_ticket;    // CTAs done; the last one resets panel_cnt and unit_ctr for the next launch
    unsigned* unit_ctr;      // next tile index (dynamic order): taken by each pair's leader as it goes
    unsigned* mode;          // this launch's tile order, set by its first CTA: 1 static, 2 dynamic
    // Several problems of different sizes in one launch (heterogeneous batches): ngroups > 0
    // chains in global memory, one per group (its own maps, shapes, scalars and panel
    // counters; same stage count); the units are stage-major across groups: ubase[s * ngroups
    // + g] is the first unit of stage s of group g and ubase[ns * ngroups] the unit count.
    // This chain then holds only the launch-level fields (ns, end_ticket, unit_ctr, mode).
    const GemmChain* groups;
    const int* ubase;
    int ngroups;
};

// One unit (pair tile) of a launch, resolved to its group's chain (C: the group's
// descriptor in global memory; unused by a single-chain launch, which reads its own
// parameters directly).
struct UnitRef {
    const GemmChain* C;
    int stg, inst, r, ntn, ntm, per_inst;
};

template <bool MULTI>
__device__ __forceinline__ UnitRef resolve_unit(const GemmChain& ch, int u) {
    UnitRef x;
    int t;
    if constexpr (!MULTI) {
        x.C = nullptr;
        x.ntn = (ch.g[0].N + 255) / 256;
        x.ntm = (ch.g[0].M + 255) / 256;
        x.per_inst = x.ntn * x.ntm;
        const int total = x.per_inst * ch.g[0].batch;
        x.stg = u / total;
        t = u - x.stg * total;
    } else {   // the last base <= u (bases are non-decreasing)
        int lo = 0, hi = ch.ns * ch.ngroups - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(ch.ubase + mid) <= u) lo = mid;
            else hi = mid - 1;
        }
        x.stg = lo / ch.ngroups;
        x.C = ch.groups + (lo - x.stg * ch.ngroups);
        x.ntn = (x.C->g[0].N + 255) / 256;
        x.ntm = (x.C->g[0].M + 255) / 256;
        x.per_inst = x.ntn * x.ntm;
        t = u - __ldg(ch.ubase + lo);
    }
    x.inst = t / x.per_inst;
    x.r = t - x.inst * x.per_inst;
    return x;
}

// The chain a unit belongs to: the launch's own parameters (constant bank) for a single
// chain, the group's descriptor otherwise.
template <bool MULTI>
__device__ __forceinline__ const GemmChain& chain_of(const GemmChain& ch, const UnitRef& x) {
    if constexpr (MULTI) return *x.C;
    else return ch;
}

// Chain launches in flight on this device (all handles).  A launch walks the static
// round-robin order only when it is the only one: the static order needs its pairs to
// become resident eventually, which holds when every other launch is either a plain
// kernel or a chain in dynamic order (neither waits on anything that is not running).
__device__ unsigned g_chain_inflight;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void mbar_arrive_local(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, int v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

// Bounded wait on an mbarrier phase with cluster-scope acquire.
__device__ __forceinline__ bool pwait_cl(uint32_t a, uint32_t parity, volatile int* abort) {
    if (mbar_try_cl(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_cl(a, parity)) {
        if (*abort) return false;
        if (gtimer() - t0 > WAIT_LIMIT_NS) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// Bounded wait until *c >= need; raises the CTA's abort flag on timeout.
__device__ __noinline__ bool panel_wait(const unsigned* c, unsigned need, volatile int* abort) {
    if (ld_acquire_u32(c) >= need) return true;
    const unsigned long long t0 = gtimer();
    while (ld_acquire_u32(c) < need) {
        if (*abort) return false;
        if (gtimer() - t0 > WAIT_LIMIT_NS) {
            *abort = 1;
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

template <int KIND, bool MULTI>
__global__ void __launch_bounds__(P_THREADS, 1) k_gemm_2sm(const __grid_constant__ GemmChain ch) {
    const GemmArgs& g0 = ch.g[0];
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    PBars2* pb = reinterpret_cast<PBars2*>(smem + ST2 * STAGE2_BYTES);
    volatile int* abort_flag = &pb->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cr = (int)cluster_rank();
    const bool leader = cr == 0;
    const int cid = blockIdx.x / 2, ncl = gridDim.x / 2;
    const int units = MULTI ? ch.ubase[ch.ns * ch.ngroups]
                            : ((g0.N + 255) / 256) * ((g0.M + 255) / 256) * g0.batch * ch.ns;
    constexpr int BK = 128 / (KIND == 0 ? 4 : 2);
    auto bar_addr = [&](uint64_t* b) { return smem_u32(b); };

    auto active = [&](const UnitRef& x) {
        const GemmArgs& a0 = chain_of<MULTI>(ch, x).g[0];
        return !a0.sc || a0.sc[x.inst].active;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST2; ++s) {
            mbar_init(bar_addr(&pb->full[s]), 1);
            mbar_init(bar_addr(&pb->empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_addr(&pb->tfull[b]), 1);
            mbar_init(bar_addr(&pb->tempty[b]), 8);   // 4 epilogue warps in each CTA
        }
        for (int k = 0; k < NU; ++k) {
            mbar_init(bar_addr(&pb->ufull[k]), 1);
            // consumers of a slot: leader's MMA thread and 4 epilogue warps, partner's producer and 4 epilogue warps
            mbar_init(bar_addr(&pb->uempty[k]), 10);
        }
        pb->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // tile order of a chain launch: decided once by its first CTA, read by the others
        if (leader && ch.ns > 1 && ch.mode) {
            unsigned m = ld_acquire_u32(ch.mode);
            if (m == 0u) {
                const unsigned prev = atomicAdd(&g_chain_inflight, 1u);
                const unsigned want = prev == 0u ? 1u : 2u;
                const unsigned old = atomicCAS(ch.mode, 0u, want);
                if (old != 0u) {
                    atomicSub(&g_chain_inflight, 1u);   // another CTA decided first
                    m = old;
                } else {
                    m = want;
                }
            }
            pb->mode = (int)m;
            st_cluster_u32(mapa_shared(smem_u32(&pb->mode), 1), (int)m);   // the partner's copy
        }
    }
    if (warp == 5) {   // joint allocation: one warp in each CTA of the pair
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&pb->tmem_slot)),
                     "r"(TMEM_COLS_P)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    cluster_sync_all();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = pb->tmem_slot;
    // Dynamic order: the leader's producer takes the next index from a global counter and
    // publishes it to every role of both CTAs through the unit ring; a dependency wait is
    // then always on smaller, already-taken tiles of running pairs.  Static order (single
    // GEMMs, and a chain alone on the device): round-robin.
    const bool dyn = ch.ns > 1 && ch.unit_ctr != nullptr && ch.mode != nullptr && pb->mode == 2;

    if (warp == 4) {
        if (lane == 0) {   // ---- TMA producer (both CTAs): own halves of A and B
            if constexpr (!MULTI)
                for (int st = 0; st < ch.ns; ++st) {
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ch.mA[st])) : "memory");
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ch.mB[st])) : "memory");
                }
            int it = 0;
            // The leader publishes tile j + 1 as it starts tile j, so that the partner (and
            // the counter's round trip) never hold up the start of a tile.
            auto publish = [&](int jj, int uu) -> bool {
                const int k = jj % NU;
                if (jj >= NU && !pwait_cl(bar_addr(&pb->uempty[k]), ((uint32_t)(jj / NU) & 1u) ^ 1u, abort_flag))
                    return false;
                pb->uslot[k] = uu;
                mbar_arrive_local(bar_addr(&pb->ufull[k]));
                st_cluster_u32(mapa_shared(smem_u32(&pb->uslot[k]), 1), uu);
                mbar_arrive_cluster(mapa_shared(bar_addr(&pb->ufull[k]), 1));
                return true;
            };
            int u_pub = 0;   // leader: the index published for the current tile
            if (dyn && leader) {
                u_pub = (int)atomicAdd(ch.unit_ctr, 1u);
                if (!publish(0, u_pub)) u_pub = units;   // abort raised: nothing to do
            }
            for (int j = 0;; ++j) {
                int u;
                if (dyn) {
                    const int k = j % NU;
                    const uint32_t ph = (uint32_t)(j / NU) & 1u;
                    if (leader) {   // tile j was published; take and publish tile j + 1
                        u = u_pub;
                        if (u < units && !*abort_flag) {
                            u_pub = (int)atomicAdd(ch.unit_ctr, 1u);
                            if (!publish(j + 1, u_pub)) break;
                        }
                    } else {
                        if (!pwait_cl(bar_addr(&pb->ufull[k]), ph, abort_flag)) break;
                        u = *reinterpret_cast<volatile int*>(&pb->uslot[k]);
                        mbar_arrive_cluster(mapa_shared(bar_addr(&pb->uempty[k]), 0));
                    }
                } else {
                    u = cid + j * ncl;
                }
                if (u >= units || *abort_flag) break;
                const UnitRef x = resolve_unit<MULTI>(ch, u);
                const GemmChain& C = chain_of<MULTI>(ch, x);
                const int stg = x.stg, inst = x.inst, r = x.r, ntn = x.ntn;
                const GemmArgs& g = C.g[stg];
                if (!active(x)) continue;
                if (C.dep[stg] && C.panel_cnt) {   // the operand panel written by the previous stage
                    const int pan = C.dep[stg] == 2 ? r % ntn : r / ntn;
                    const unsigned* c = C.panel_cnt + ((size_t)(stg - 1) * C.g[0].batch + inst) * x.ntm + pan;
                    if (!panel_wait(c, 8u * (unsigned)ntn, abort_flag)) break;
                    asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes -> TMA reads
                }
                const CUtensorMap* mA = &C.mA[stg];
                const CUtensorMap* mB = &C.mB[stg];
                const int m0 = (r / ntn) * 256 + cr * 128, nh = (r % ntn) * 256 + cr * 128;
                const int za = g.a_shared ? 0 : inst, zb = g.b_shared ? 0 : inst;
                for (int kb = 0; kb < g.nk; ++kb, ++it) {
                    const int s = it % ST2;
                    const uint32_t ph = (uint32_t)(it / ST2) & 1u;
                    if (it >= ST2 && !pwait(bar_addr(&pb->empty[s]), ph ^ 1u, abort_flag)) break;
                    const uint32_t sa = smem_u32(smem + s * STAGE2_BYTES);
                    const uint32_t fl = mapa_shared(bar_addr(&pb->full[s]), 0);
                    if (leader) mbar_expect_tx(bar_addr(&pb->full[s]), 2 * STAGE2_BYTES);   // both CTAs' halves
                    tma_load_3d_pair(sa, mA, fl, kb * BK, m0, za);
                    tma_load_3d_pair(sa + A2_BYTES, mB, fl, kb * BK, nh, zb);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0 && leader) {   // ---- MMA issuer (leader CTA only)
            int it = 0, tl = 0;
            for (int j = 0;; ++j) {
                int u;
                if (dyn) {
                    const int k = j % NU;
                    if (!pwait_cl(bar_addr(&pb->ufull[k]), (uint32_t)(j / NU) & 1u, abort_flag)) break;
                    u = *reinterpret_cast<volatile int*>(&pb->uslot[k]);
                    mbar_arrive_cluster(mapa_shared(bar_addr(&pb->uempty[k]), 0));
                } else {
                    u = cid + j * ncl;
                }
                if (u >= units || *abort_flag) break;
                const UnitRef x = resolve_unit<MULTI>(ch, u);
                if (!active(x)) continue;
                const int nk = chain_of<MULTI>(ch, x).g[0].nk;
                const int b = tl & 1;
                const uint32_t use = (uint32_t)(tl >> 1);
                if (tl >= 2 && !pwait(bar_addr(&pb->tempty[b]), (use - 1u) & 1u, abort_flag)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * 256);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = it % ST2;
                    const uint32_t ph = (uint32_t)(it / ST2) & 1u;
                    if (!pwait(bar_addr(&pb->full[s]), ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(smem + s * STAGE2_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma2<KIND>(d, make_desc(sa + 32 * kk), make_desc(sa + A2_BYTES + 32 * kk), (kb | kk) != 0);
                    commit2_mc(bar_addr(&pb->empty[s]), 3);   // stage free in both CTAs
                }
                commit2_mc(bar_addr(&pb->tfull[b]), 3);       // accumulator ready in both CTAs
                ++tl;
                if (!ok) break;
            }
        }
    } else {   // ---- epilogue warps 0-3 (both CTAs): thread = TMEM lane = output row
        int tl = 0;
        int nst = 0;   // TMA stores this warp has issued (staging buffers alternate)
        uint8_t* stage = reinterpret_cast<uint8_t*>(
            (reinterpret_cast<uintptr_t>(smem + ST2 * STAGE2_BYTES + sizeof(PBars2)) + 1023) & ~(uintptr_t)1023);
        for (int j = 0;; ++j) {
            int u;
            if (dyn) {
                const int k = j % NU;
                int uu = 0, okw = 1;
                if (lane == 0) {
                    okw = pwait_cl(bar_addr(&pb->ufull[k]), (uint32_t)(j / NU) & 1u, abort_flag) ? 1 : 0;
                    if (okw) {
                        uu = *reinterpret_cast<volatile int*>(&pb->uslot[k]);
                        mbar_arrive_cluster(mapa_shared(bar_addr(&pb->uempty[k]), 0));
                    }
                }
                okw = __shfl_sync(0xffffffffu, okw, 0);
                uu = __shfl_sync(0xffffffffu, uu, 0);
                if (!okw) break;
                u = uu;
            } else {
                u = cid + j * ncl;
            }
            if (u >= units) break;
            const UnitRef x = resolve_unit<MULTI>(ch, u);
            const GemmChain& C = chain_of<MULTI>(ch, x);
            const int stg = x.stg, inst = x.inst, r = x.r, ntn = x.ntn;
            const GemmArgs& g = C.g[stg];
            if (!active(x)) continue;
            const int cta_per_inst = x.per_inst * 2;
            const int m0 = (r / ntn) * 256 + cr * 128, n0 = (r % ntn) * 256;
            const int ct = ((r / ntn) * 2 + cr) * ntn + (r % ntn);
            const int b = tl & 1;
            const uint32_t use = (uint32_t)(tl >> 1);
            const bool ok = pwait(bar_addr(&pb->tfull[b]), use & 1u, abort_flag);
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = m0 + warp * 32 + lane;
            const bool m_ok = m < g.M;
            const int epi = g.epi;
            float mu_m = 0.f;
            if (epi == EPI_DIV && m_ok) mu_m = g.mu[m];
            const float inv_scale = (epi == EPI_Z && g.scl) ? (float)(1.0 / g.scl[inst].rscale) : 1.f;
            double acc = 0.0;
            const uint32_t tm = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 256);
            const bool tma_out = C.ostore[stg] != 0;
            if (tma_out) {
                const CUtensorMap* om = &C.mO[stg];
                const int mw = m0 + warp * 32;
                if (epi == EPI_DIV)
                    epi_tile_tma<EPI_DIV, KIND>(g, om, tm, inst, m, m_ok, mw, n0, mu_m, inv_scale, acc, stage, warp,
                                                lane, nst);
                else if (epi == EPI_Z)
                    epi_tile_tma<EPI_Z, 0>(g, om, tm, inst, m, m_ok, mw, n0, mu_m, inv_scale, acc, stage, warp, lane,
                                           nst);
                else
                    epi_tile_tma<EPI_STORE, KIND>(g, om, tm, inst, m, m_ok, mw, n0, mu_m, inv_scale, acc, stage,
                                                  warp, lane, nst);
            } else {
#pragma unroll 1
                for (int c = 0; c < 256 / 32; ++c) {
                    float v[32];
                    tmem_ld32(tm + (uint32_t)(c * 32), v);
                    const int nb = n0 + c * 32;
                    if (m_ok && nb < g.N) {
                        if (epi == EPI_DIV) epi_chunk<EPI_DIV, KIND>(g, inst, m, nb, v, mu_m, inv_scale, acc);
                        else if (epi == EPI_Z) epi_chunk<EPI_Z, 0>(g, inst, m, nb, v, mu_m, inv_scale, acc);
                        else epi_chunk<EPI_STORE, KIND>(g, inst, m, nb, v, mu_m, inv_scale, acc);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(mapa_shared(bar_addr(&pb->tempty[b]), 0));
            if (stg + 1 < C.ns && C.dep[stg + 1] && C.panel_cnt) {
                // publish this warp's 32 rows of the tile to the next stage's TMA reads
                // (4 warps x 2 CTAs per tile: a panel of ntn tiles is complete at 8 ntn);
                // TMA-stored rows first complete their stores
                if (tma_out) {
                    if (lane == 0) bulk_wait_all();
                    __syncwarp();
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicAdd(C.panel_cnt + ((size_t)stg * C.g[0].batch + inst) * x.ntm + r / ntn, 1u);
            }
            if (epi == EPI_Z && g.rz_part) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) pb->red[tl & 1][warp] = acc;
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (warp == 0) {
                    int last = 0;
                    if (lane == 0) {
                        const double* rd = pb->red[tl & 1];
                        g.rz_part[(size_t)inst * cta_per_inst + ct] = rd[0] + rd[1] + rd[2] + rd[3];
                        if (g.sc && g.counter) {
                            __threadfence();
                            const unsigned tk = atomicAdd(g.counter + inst, 1u);
                            last = (tk == (unsigned)cta_per_inst - 1) ? 1 : 0;
                        }
                    }
                    last = __shfl_sync(0xffffffffu, last, 0);
                    if (last) {   // fixed-order sum of this instance's partials: rz and beta
                        __threadfence();
                        double rz = 0.0;
                        for (int i = lane; i < cta_per_inst; i += 32)
                            rz += __ldcg(g.rz_part + (size_t)inst * cta_per_inst + i);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) rz += __shfl_xor_sync(0xffffffffu, rz, o);
                        if (lane == 0) {
                            g.counter[inst] = 0;
                            PcgScalars* p = g.sc + inst;
                            double beta = (rz - (g.flex ? p->rzo : 0.0)) / p->rz;
                            if (!isfinite(beta)) beta = 0.0;
                            p->beta = beta;
                            p->rz = rz;
                        }
                    }
                }
            }
            ++tl;
        }
        if (lane == 0) bulk_wait_all();   // staged rows stored before the shared memory is released
    }
    __syncthreads();
    cluster_sync_all();   // the peer's copies, commits and arrivals have all landed
    if (threadIdx.x == 0 && pb->abort) {
        if (MULTI)
            for (int gi = 0; gi < ch.ngroups; ++gi) {
                if (ch.groups[gi].g[0].status) atomicOr(ch.groups[gi].g[0].status, DEV_ERR_TIMEOUT);
            }
        else if (g0.status)
            atomicOr(g0.status, DEV_ERR_TIMEOUT);
    }
    if (threadIdx.x == 0 && (ch.panel_cnt || ch.ngroups) && ch.ns > 1) {
        __threadfence();
        const unsigned tk = atomicAdd(ch.end_ticket, 1u);
        if (tk == gridDim.x - 1) {   // every CTA is done with the counters: reset them
            const int ng = MULTI ? ch.ngroups : 1;
            for (int gi = 0; gi < ng; ++gi) {
                const GemmChain& C = MULTI ? ch.groups[gi] : ch;
                if (!C.panel_cnt) continue;
                const int ncnt = (C.ns - 1) * C.g[0].batch * ((C.g[0].M + 255) / 256);
                for (int i = 0; i < ncnt; ++i) C.panel_cnt[i] = 0u;
            }
            if (ch.unit_ctr) *ch.unit_ctr = 0u;
            if (ch.mode) {   // the launch's registration in the in-flight count ends here
                *ch.mode = 0u;
                atomicSub(&g_chain_inflight, 1u);
            }
            *ch.end_ticket = 0u;
            __threadfence();
        }
    }
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS_P) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {   // thread-safe one-time lookup
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

// 3D tensor map over [batch][rows][cols] (cols contiguous, leading dimension ld),
// box = 128 bytes of K x box_rows rows x 1 instance, 128-byte swizzle.
mofem_status make_map(CUtensorMap* m, const void* base, int esize, int cols, int rows, int batch, int ld,
                      int box_rows, bool fp16 = false) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        mofem_set_last_error("cuTensorMapEncodeTiled entry point unavailable", __FILE__, __LINE__);
        return MOFEM_ERR_CUDA;
    }
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)ld * esize, (cuuint64_t)rows * ld * esize};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    CUresult r = enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[96];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        mofem_set_last_error(buf, __FILE__, __LINE__);
        return MOFEM_ERR_CUDA;
    }
    return MOFEM_OK;
}

}  // namespace

// 3D tensor map over [batch][rows][cols] for plain (unswizzled) row tiles of
// box_cols x box_rows elements (the operator-apply staging).
mofem_status make_row_map(CUtensorMap* m, const void* base, int esize, int cols, int rows, int batch, int ld,
                          int box_cols, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        mofem_set_last_error("cuTensorMapEncodeTiled entry point unavailable", __FILE__, __LINE__);
        return MOFEM_ERR_CUDA;
    }
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)ld * esize, (cuuint64_t)rows * ld * esize};
    cuuint32_t box[3] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        char buf[96];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled (rows) failed (%d)", (int)r);
        mofem_set_last_error(buf, __FILE__, __LINE__);
        return MOFEM_ERR_CUDA;
    }
    return MOFEM_OK;
}

namespace {

int num_sms() {
    static std::atomic<int> cache[MOFEM_MAX_DEV];
    const int slot = dev_slot();
    int n = cache[slot].load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
        cache[slot].store(n, std::memory_order_relaxed);
    }
    return n;
}

constexpr int GEMM_CM = 2;   // CTAs per cluster: one tcgen05 CTA pair

template <int KIND, bool MULTI>
mofem_status launch_chain(const GemmChain& ch0, int batch, cudaStream_t st) {
    constexpr int CM = GEMM_CM;
    auto kern = k_gemm_2sm<KIND, MULTI>;
    static std::atomic<int> max_pairs_dev[MOFEM_MAX_DEV];   // per device: co-resident pairs
    std::atomic<int>& max_pairs_slot = max_pairs_dev[dev_slot()];
    int max_pairs = max_pairs_slot.load(std::memory_order_acquire);
    const int smem = ST2 * STAGE2_BYTES + 1024 + (int)sizeof(PBars2) + 1024 + EPI_STAGE_TOTAL;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CM;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (!max_pairs) {
        MOFEM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        cfg.gridDim = dim3(CM * (num_sms() / CM));
        int n = 0;
        MOFEM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, kern, &cfg));
        if (n <= 0) {
            mofem_set_last_error("no CTA pair of the tensor-core GEMM fits on this GPU", __FILE__, __LINE__);
            return MOFEM_ERR_UNSUPPORTED;
        }
        max_pairs = n;
        max_pairs_slot.store(n, std::memory_order_release);
    }
    GemmChain ch = ch0;
    if (MULTI != (ch.ngroups > 0)) return MOFEM_ERR_INVALID_ARG;
    if (MULTI) {   // heterogeneous launch: descriptors validated when they were built
        if (!ch.groups || !ch.ubase || !ch.end_ticket || !ch.unit_ctr || !ch.mode || batch <= 0)
            return MOFEM_ERR_INVALID_ARG;
        const int pairs = batch < max_pairs ? batch : max_pairs;   // batch = the launch's unit count
        cfg.gridDim = dim3(CM * pairs);
        MOFEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, ch));
        return MOFEM_OK;
    }
    if (ch.ns < 1 || ch.ns > CHAIN_MAX ||
        (ch.ns > 1 && (!ch.panel_cnt || !ch.end_ticket || !ch.unit_ctr || !ch.mode)))
        return MOFEM_ERR_INVALID_ARG;
    if (ch.ns > 1 && ch.g[0].M != ch.g[0].N) return MOFEM_ERR_INVALID_ARG;   // panels index rows and columns alike
    for (int s = 0; s < ch.ns; ++s) {
        GemmArgs& g = ch.g[s];
        g.batch = batch;
        // output type follows the operand kind (FP32 for TF32, BF16, FP16), except G4's FP32 Z;
        // every stage shares the first one's shape and scalar state
        if (g.out_bf16 != (g.epi == EPI_Z ? 0 : KIND)) return MOFEM_ERR_INVALID_ARG;
        if (g.M != ch.g[0].M || g.N != ch.g[0].N || g.nk != ch.g[0].nk || g.sc != ch.g[0].sc) return MOFEM_ERR_INVALID_ARG;
        if (s == 0 ? ch.dep[s] != 0 : (ch.dep[s] < 0 || ch.dep[s] > 2)) return MOFEM_ERR_INVALID_ARG;
    }
    for (int s = ch.ns; s < CHAIN_MAX; ++s) ch.dep[s] = 0;
    const int total = ((ch.g[0].N + BN - 1) / BN) * ((ch.g[0].M + BM * CM - 1) / (BM * CM)) * batch;   // pair tiles
    const int units = total * ch.ns;
    const int pairs = units < max_pairs ? units : max_pairs;
    cfg.gridDim = dim3(CM * pairs);
    MOFEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, ch));
    return MOFEM_OK;
}

mofem_status launch_chain_kind(int which, const GemmChain& ch, int batch, cudaStream_t st) {
    if (ch.ngroups > 0) {
        if (which == 1) return launch_chain<1, true>(ch, batch, st);
        if (which == 2) return launch_chain<2, true>(ch, batch, st);
        return launch_chain<0, true>(ch, batch, st);
    }
    if (which == 1) return launch_chain<1, false>(ch, batch, st);
    if (which == 2) return launch_chain<2, false>(ch, batch, st);
    return launch_chain<0, false>(ch, batch, st);
}

// One GEMM: a chain of one stage.
mofem_status launch_single(int which, const CUtensorMap& mA, const CUtensorMap& mB, const GemmArgs& g, int batch,
                           cudaStream_t st) {
    GemmChain ch{};
    ch.mA[0] = mA;
    ch.mB[0] = mB;
    ch.g[0] = g;
    ch.ns = 1;
    return launch_chain_kind(which, ch, batch, st);
}

}  // namespace

mofem_status launch_transpose64_ld(const double* src, long long s_bs, int s_ld, double* dst, long long d_bs, int d_ld,
                                   int n, int batch, cudaStream_t st);

mofem_status launch_gemm_kind(int which, const CUtensorMap& mA, const CUtensorMap& mB, const GemmArgs& g, int batch,
                              cudaStream_t st) {
    return launch_single(which, mA, mB, g, batch, st);
}

// <R, Z> partial slots per instance: one per CTA tile of the paired grid
int tc_rz_ctas(const mofem_ctx* c) {
    return ((c->q + BN - 1) / BN) * ((c->q + BM * GEMM_CM - 1) / (BM * GEMM_CM)) * GEMM_CM;
}

// Allocate the operand copies of Q1, Q1^T, Q2, Q2^T in the precision `which`
// (0 TF32 = FP32 storage, 1 BF16), the intermediates, and the tensor maps.
mofem_status tc_prepare(mofem_ctx* c, int which, cudaStream_t st) {
    TcPlan& p = c->tc[which];
    if (p.ready) return MOFEM_OK;
    const int q = c->q, ld = c->ld, B = c->batch;
    const int es = which == 0 ? 4 : 2;
    const int kind = conv_kind_of_plan(which);   // launch_convert kinds: 0 float, 2 bf16, 3 f16
    const bool f16 = which == 2;
    p.esize = es;
    const size_t per = (size_t)q * ld;
    MOFEM_CUDA_TRY(cudaMalloc(&p.Q1, per * B * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.Q1T, per * B * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.Q2, per * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.Q2T, per * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.Rop, per * B * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.X1T, per * B * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.WT, per * B * es));
    MOFEM_CUDA_TRY(cudaMalloc(&p.Y, per * B * es));
    void* zero[] = {p.Q1, p.Q1T, p.Rop, p.X1T, p.WT, p.Y};
    for (void* z : zero) MOFEM_CUDA_TRY(cudaMemsetAsync(z, 0, per * B * es, st));
    MOFEM_CUDA_TRY(cudaMemsetAsync(p.Q2, 0, per * es, st));
    MOFEM_CUDA_TRY(cudaMemsetAsync(p.Q2T, 0, per * es, st));
    // panel counters of the GEMM chain (three producing stages) and its end ticket, self-resetting
    p.n_panel_cnt = 3 * B * ((q + 255) / 256);
    // + end ticket, unit counter, order word
    MOFEM_CUDA_TRY(cudaMalloc(&p.panel_cnt, sizeof(unsigned) * (p.n_panel_cnt + 3)));
    MOFEM_CUDA_TRY(cudaMemsetAsync(p.panel_cnt, 0, sizeof(unsigned) * (p.n_panel_cnt + 3), st));
    double* tmp = nullptr;
    MOFEM_CUDA_TRY(cudaMalloc(&tmp, per * sizeof(double)));
    MOFEM_TRY(launch_convert(c->Q2_64, 1, per, ld, p.Q2, kind, per, ld, q, q, 1, st));
    MOFEM_TRY(launch_transpose64_ld(c->Q2_64, per, ld, tmp, per, ld, q, 1, st));
    MOFEM_TRY(launch_convert(tmp, 1, per, ld, p.Q2T, kind, per, ld, q, q, 1, st));
    for (int i = 0; i < B; ++i) {
        const double* q1 = c->Q1_64 + per * i;
        MOFEM_TRY(launch_convert(q1, 1, per, ld, (char*)p.Q1 + per * i * es, kind, per, ld, q, q, 1, st));
        MOFEM_TRY(launch_transpose64_ld(q1, per, ld, tmp, per, ld, q, 1, st));
        MOFEM_TRY(launch_convert(tmp, 1, per, ld, (char*)p.Q1T + per * i * es, kind, per, ld, q, q, 1, st));
    }
    MOFEM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(tmp);
    // A maps and B maps (box rows BM = BN / 2: B slices arrive in two halves) of the four GEMMs
    MOFEM_TRY(make_map(&p.mA[0], p.Q2T, es, q, q, 1, ld, BM, f16));
    MOFEM_TRY(make_map(&p.mB[0], p.Rop, es, q, q, B, ld, BN / 2, f16));
    MOFEM_TRY(make_map(&p.mA[1], p.X1T, es, q, q, B, ld, BM, f16));
    MOFEM_TRY(make_map(&p.mB[1], p.Q1T, es, q, q, B, ld, BN / 2, f16));
    MOFEM_TRY(make_map(&p.mA[2], p.Q1, es, q, q, B, ld, BM, f16));
    MOFEM_TRY(make_map(&p.mB[2], p.WT, es, q, q, B, ld, BN / 2, f16));
    MOFEM_TRY(make_map(&p.mA[3], p.Y, es, q, q, B, ld, BM, f16));
    MOFEM_TRY(make_map(&p.mB[3], p.Q2, es, q, q, 1, ld, BN / 2, f16));
    // output maps of the TMA-store epilogue: 32-row boxes of one 128-byte swizzled row block
    MOFEM_TRY(make_map(&p.mO[0], p.X1T, es, q, q, B, ld, 32, f16));
    MOFEM_TRY(make_map(&p.mO[1], p.WT, es, q, q, B, ld, 32, f16));
    MOFEM_TRY(make_map(&p.mO[2], p.Y, es, q, q, B, ld, 32, f16));
    p.ready = true;
    return MOFEM_OK;
}

// One of the four GEMMs (index 0..3) on the plan's internal buffers (timing).
mofem_status tc_gemm_one(const mofem_ctx* c, int which, int idx, float* Z, cudaStream_t st) {
    const TcPlan& p = c->tc[which];
    const int q = c->q, ld = c->ld;
    const int bk = which == 0 ? 32 : 64;
    GemmArgs g{};
    g.M = q; g.N = q; g.nk = (q + bk - 1) / bk;
    g.status = c->d_status;
    g.lam = c->lam32; g.lam_bs = ld; g.mu = c->mu32; g.div_product = c->div_product;
    g.out_bs = (long long)q * ld; g.out_ld = ld; g.out_bf16 = which;
    g.pad_ok = 1;   // internal buffers, zero padding
    void* outs[4] = {p.X1T, p.WT, p.Y, Z};
    const int epis[4] = {EPI_STORE, EPI_DIV, EPI_STORE, EPI_Z};
    g.out = outs[idx]; g.epi = epis[idx];
    g.a_shared = idx == 0; g.b_shared = idx == 3;
    if (idx == 3) g.out_bf16 = 0;
    return launch_gemm_kind(which, p.mA[idx], p.mB[idx], g, c->batch, st);
}

// The four-stage chain of Z = P^{-1}(R) with R already in p.Rop (rounded operand).
// R32 (FP32, same layout as Z) feeds the fused <R, Z> partials when rz_partial != nullptr.
static GemmChain tc_chain(const mofem_ctx* c, int which, const float* R32, long long r_bs, int r_ld, float* Z, int z_ld,
                   long long z_bs, double* rz_partial, PcgScalars* sc, bool z_internal) {
    const TcPlan& p = c->tc[which];
    const int q = c->q, ld = c->ld;
    const int bk = which == 0 ? 32 : 64;
    GemmArgs g{};
    g.M = q;
    g.N = q;
    g.nk = (q + bk - 1) / bk;
    g.sc = sc;
    g.status = c->d_status;
    g.lam = c->lam32;
    g.lam_bs = ld;
    g.mu = c->mu32;
    g.div_product = c->div_product;
    g.out_bs = (long long)q * ld;
    g.out_ld = ld;
    g.out_bf16 = which;
    g.scl = which == 2 ? c->d_sc : nullptr;
    g.pad_ok = 1;   // G1..G3 write internal intermediates
    GemmChain ch{};
    for (int i = 0; i < 4; ++i) {
        ch.mA[i] = p.mA[i];
        ch.mB[i] = p.mB[i];
    }
    // G1: X1T = (R Q2)^T
    g.out = p.X1T; g.epi = EPI_STORE; g.a_shared = 1; g.b_shared = 0;
    ch.g[0] = g;
    // G2: WT[j][i] = (Q1^T X1)[i][j] / (lam_i + mu_j)   (A = X1T: rows written by G1)
    g.out = p.WT; g.epi = EPI_DIV; g.a_shared = 0; g.b_shared = 0;
    ch.g[1] = g; ch.dep[1] = 1;
    // G3: Y = Q1 W   (B = WT: rows written by G2)
    g.out = p.Y; g.epi = EPI_STORE; g.a_shared = 0; g.b_shared = 0;
    ch.g[2] = g; ch.dep[2] = 2;
    // G4: Z = Y Q2^T (+ <R, Z> partials)   (A = Y: rows written by G3)
    g.out = Z; g.out_bs = z_bs; g.out_ld = z_ld; g.out_bf16 = 0; g.epi = EPI_Z; g.a_shared = 0; g.b_shared = 1;
    g.pad_ok = z_internal ? 1 : 0;   // a caller's Z keeps its padding untouched
    g.R = R32; g.r_bs = r_bs; g.r_ld = r_ld; g.rz_part = rz_partial;
    g.counter = c->d_ctr + 2 * c->batch;
    g.flex = 1;
    ch.g[3] = g; ch.dep[3] = 1;
    ch.ns = 4;
    ch.panel_cnt = p.panel_cnt;
    ch.end_ticket = p.panel_cnt + p.n_panel_cnt;
    ch.unit_ctr = p.panel_cnt + p.n_panel_cnt + 1;
    ch.mode = p.panel_cnt + p.n_panel_cnt + 2;
    for (int s = 0; s < 4; ++s) ch.g[s].batch = c->batch;
    // TMA-store epilogue: the intermediates always; Z where its rows are 16-byte aligned
    for (int s = 0; s < 3; ++s) {
        ch.mO[s] = p.mO[s];
        ch.ostore[s] = 1;
    }
    const bool z_aligned = (reinterpret_cast<uintptr_t>(Z) % 16) == 0 && ((long long)z_ld * 4) % 16 == 0 &&
                           (z_bs * 4) % 16 == 0 && z_bs == (long long)z_ld * q;
    ch.ostore[3] = (z_aligned && make_map(&ch.mO[3], Z, 4, q, q, c->batch, z_ld, 32) == MOFEM_OK) ? 1 : 0;
    return ch;
}

mofem_status tc_precond(const mofem_ctx* c, int which, const float* R32, long long r_bs, int r_ld, float* Z, int z_ld,
                        long long z_bs, double* rz_partial, PcgScalars* sc, cudaStream_t st, bool z_internal) {
    return launch_chain_kind(which, tc_chain(c, which, R32, r_bs, r_ld, Z, z_ld, z_bs, rz_partial, sc, z_internal),
                             c->batch, st);
}

// ---- heterogeneous launches: the chains of several handles (any q) in one persistent launch
mofem_status tc_multi_build(const TcGroupArgs* ga, int n, int which, TcMulti* out) {
    *out = TcMulti{};
    if (n < 1) return MOFEM_ERR_INVALID_ARG;
    std::vector<GemmChain> chains(n);
    std::vector<const mofem_ctx*> cs(n);
    for (int gi = 0; gi < n; ++gi) {
        const mofem_ctx* c = ga[gi].c;
        cs[gi] = c;
        if (!c->tc[which].ready) return MOFEM_ERR_INVALID_ARG;
        const long long bs = (long long)c->q * c->ld;
        chains[gi] = tc_chain(c, which, ga[gi].R32, bs, c->ld, ga[gi].Z, c->ld, bs, ga[gi].rz_partial, c->d_sc, true);
    }
    std::vector<int> ubase((size_t)4 * n + 1, 0);
    int run = 0;
    for (int s = 0; s < 4; ++s)
        for (int gi = 0; gi < n; ++gi) {
            ubase[(size_t)s * n + gi] = run;
            const GemmArgs& g = chains[gi].g[0];
            if (chains[gi].ns != 4 || g.M != g.N || g.batch != cs[gi]->batch) return MOFEM_ERR_INVALID_ARG;
            run += ((g.N + BN - 1) / BN) * ((g.M + BM * GEMM_CM - 1) / (BM * GEMM_CM)) * g.batch;
        }
    ubase[(size_t)4 * n] = run;
    out->ngroups = n;
    out->units = run;
    out->which = which;
    MOFEM_CUDA_TRY(cudaMalloc(&out->d_groups, sizeof(GemmChain) * n));
    static_assert(sizeof(GemmChain) % 64 == 0, "tensor maps in the descriptor array stay 64-byte aligned");
    MOFEM_CUDA_TRY(cudaMalloc(&out->d_ubase, sizeof(int) * ubase.size()));
    MOFEM_CUDA_TRY(cudaMalloc(&out->d_ctr, sizeof(unsigned) * 3));
    MOFEM_CUDA_TRY(cudaMemcpy(out->d_groups, chains.data(), sizeof(GemmChain) * n, cudaMemcpyHostToDevice));
    MOFEM_CUDA_TRY(cudaMemcpy(out->d_ubase, ubase.data(), sizeof(int) * ubase.size(), cudaMemcpyHostToDevice));
    MOFEM_CUDA_TRY(cudaMemset(out->d_ctr, 0, sizeof(unsigned) * 3));
    return MOFEM_OK;
}

mofem_status tc_multi_launch(const TcMulti& m, cudaStream_t st) {
    GemmChain ch{};
    ch.ns = 4;
    ch.groups = static_cast<const GemmChain*>(m.d_groups);
    ch.ubase = m.d_ubase;
    ch.ngroups = m.ngroups;
    ch.end_ticket = m.d_ctr;
    ch.unit_ctr = m.d_ctr + 1;
    ch.mode = m.d_ctr + 2;
    return launch_chain_kind(m.which, ch, m.units, st);
}

void tc_multi_free(TcMulti* m) {
    cudaFree(m->d_groups);
    cudaFree(m->d_ubase);
    cudaFree(m->d_ctr);
    *m = TcMulti{};
}

// The four preconditioner GEMMs on caller-provided BF16 buffers (operand copies
// Q1, Q1T, Q2, Q2T; rounded R in Rop; intermediates X1T, WT, Y), all
// [batch][q][ld] (Q2, Q2T: one instance).  Builds its tensor maps on the host
// (no allocation) and writes Z (FP32, z_ld, z_bs).
mofem_status tc_precond_buffers(const mofem_ctx* c, const TcBuffers& b, float* Z, int z_ld, long long z_bs,
                                cudaStream_t st) {
    const int q = c->q, ld = b.ld, B = c->batch;
    CUtensorMap mA[4], mB[4];
    MOFEM_TRY(make_map(&mA[0], b.Q2T, 2, q, q, 1, ld, BM));
    MOFEM_TRY(make_map(&mB[0], b.Rop, 2, q, q, B, ld, BN / 2));
    MOFEM_TRY(make_map(&mA[1], b.X1T, 2, q, q, B, ld, BM));
    MOFEM_TRY(make_map(&mB[1], b.Q1T, 2, q, q, B, ld, BN / 2));
    MOFEM_TRY(make_map(&mA[2], b.Q1, 2, q, q, B, ld, BM));
    MOFEM_TRY(make_map(&mB[2], b.WT, 2, q, q, B, ld, BN / 2));
    MOFEM_TRY(make_map(&mA[3], b.Y, 2, q, q, B, ld, BM));
    MOFEM_TRY(make_map(&mB[3], b.Q2, 2, q, q, 1, ld, BN / 2));
    GemmArgs g{};
    g.M = q; g.N = q; g.nk = (q + 63) / 64;
    g.status = c->d_status;
    g.lam = c->lam32; g.lam_bs = c->ld; g.mu = c->mu32; g.div_product = c->div_product;
    g.out_bs = (long long)q * ld; g.out_ld = ld; g.out_bf16 = 1;
    g.pad_ok = 1;   // the library's own scratch array
    g.out = b.X1T; g.epi = EPI_STORE; g.a_shared = 1; g.b_shared = 0;
    MOFEM_TRY(launch_single(1, mA[0], mB[0], g, B, st));
    g.out = b.WT; g.epi = EPI_DIV; g.a_shared = 0; g.b_shared = 0;
    MOFEM_TRY(launch_single(1, mA[1], mB[1], g, B, st));
    g.out = b.Y; g.epi = EPI_STORE;
    MOFEM_TRY(launch_single(1, mA[2], mB[2], g, B, st));
    g.out = Z; g.out_bs = z_bs; g.out_ld = z_ld; g.out_bf16 = 0; g.epi = EPI_Z; g.a_shared = 0; g.b_shared = 1;
    g.pad_ok = 0;   // the caller's Z
    return launch_single(1, mA[3], mB[3], g, B, st);
}
