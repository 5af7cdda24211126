// FP32 instantiations of the banded operator apply (mixed-precision inner solve).
#include "apply_pcg_f2.cuh"
#include "apply_pcg_push.cuh"

using namespace mofem_apply_impl;

mofem_status launch_apply_f64(int K, int nt, int mode, const ApplyArgs& a, int batch, cudaStream_t st);
mofem_status launch_apply_pcg_f64(int K, int nt, const CUtensorMap& mZ, const CUtensorMap& mQ, const ApplyPcgArgs& a,
                                  int batch, cudaStream_t st);

template <int K, int NT>
static mofem_status dispatch_mode_f32(int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    switch (mode) {
        case APPLY_PLAIN: return launch_t<float, K, NT, APPLY_PLAIN, false>(a, batch, st);
        case APPLY_QUPDATE: return launch_t<float, K, NT, APPLY_QUPDATE, false>(a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

template <int K>
static mofem_status dispatch_nt_f32(int nt, int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    if (nt == 5) return dispatch_mode_f32<K, 5>(mode, a, batch, st);
    if (nt == 8) return dispatch_mode_f32<K, 8>(mode, a, batch, st);
    return MOFEM_ERR_UNSUPPORTED;
}

mofem_status launch_apply(int K, int nt, bool fp64, int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    if (a.rows_out <= 0 || a.cols_out <= 0 || batch <= 0) return MOFEM_OK;
    if (fp64) return launch_apply_f64(K, nt, mode, a, batch, st);
    switch (K) {
        case 1: return dispatch_nt_f32<1>(nt, mode, a, batch, st);
        case 2: return dispatch_nt_f32<2>(nt, mode, a, batch, st);
        case 3: return dispatch_nt_f32<3>(nt, mode, a, batch, st);
        case 4: return dispatch_nt_f32<4>(nt, mode, a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

int apply_rows_per_cta(int K) {
    switch (K) {
        case 1: return Geo<1>::TA_G;
        case 2: return Geo<2>::TA_G;
        case 3: return Geo<3>::TA_G;
        default: return Geo<4>::TA_G;
    }
}

// The streaming FP32 apply with the s-pass in push form (k_apply_pcg4) or over a register
// window of t-pass rows (k_apply_pcg3); the coefficient table of the handle follows.
constexpr bool kApplyPush = true;
bool apply_push_layout() { return kApplyPush; }

template <int K, int NT>
static mofem_status pcg_f32(const CUtensorMap& mZ, const CUtensorMap& mQ, const CUtensorMap* mS,
                           const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    if constexpr (packed_apply_ok(K, NT)) {
        if (!mS) return MOFEM_ERR_INVALID_ARG;
        if constexpr (kApplyPush) return launch_pcg4_t<K, NT>(mZ, mQ, *mS, a, batch, st);
        else return launch_pcg3_t<K, NT>(mZ, mQ, *mS, a, batch, st);
    } else {
        return launch_pcg_t<float, K, NT, false>(mZ, mQ, a, batch, st);
    }
}

template <int K>
static mofem_status pcg_nt_f32(int nt, const CUtensorMap& mZ, const CUtensorMap& mQ, const CUtensorMap* mS,
                               const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    if (nt == 5) return pcg_f32<K, 5>(mZ, mQ, mS, a, batch, st);
    if (nt == 8) return pcg_f32<K, 8>(mZ, mQ, mS, a, batch, st);
    return MOFEM_ERR_UNSUPPORTED;
}

mofem_status launch_apply_pcg(int K, int nt, bool fp64, const CUtensorMap& mZ, const CUtensorMap& mQ,
                              const CUtensorMap* mS, const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    if (fp64) return launch_apply_pcg_f64(K, nt, mZ, mQ, a, batch, st);
    switch (K) {
        case 1: return pcg_nt_f32<1>(nt, mZ, mQ, mS, a, batch, st);
        case 2: return pcg_nt_f32<2>(nt, mZ, mQ, mS, a, batch, st);
        case 3: return pcg_nt_f32<3>(nt, mZ, mQ, mS, a, batch, st);
        case 4: return pcg_nt_f32<4>(nt, mZ, mQ, mS, a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

bool apply_pcg_packed(int K, int nt, bool fp64) { return !fp64 && packed_apply_ok(K, nt); }

// Rows per CTA of the tiled PCG-form apply (FP64 and the wide FP32 forms).
int apply_pcg_rows_per_cta(int K, int nt, bool fp64) {
    (void)nt;
    (void)fp64;
    switch (K) {
        case 1: return Geo<1>::TA_T;
        case 2: return Geo<2>::TA_T;
        case 3: return Geo<3>::TA_T;
        default: return Geo<4>::TA_T;
    }
}

// Rows of one TMA box of Z / Q_prev: a staged chunk of the streaming apply, or the tile
// with its K-row halo of the tiled one.
int apply_pcg_box_rows(int K, int nt, bool fp64) {
    if (apply_pcg_packed(K, nt, fp64)) return Geo3<2, 5, 1>::CR;
    return apply_pcg_rows_per_cta(K, nt, fp64) + 2 * K;
}

// Rows of one TMA box of the S rows (streaming apply).
int apply_pcg_s_box_rows() { return Geo3<2, 5, 1>::CR; }

// SR of Geo3 / Geo4: floats per coefficient row, NT (2K + 1) padded to a multiple of 8
int apply_s_row_floats(int K, int nt) { return ((nt * (2 * K + 1) + 7) / 8) * 8; }

// (the largest tile-height divisor the handles use: partial slots are sized for it)
constexpr int APPLY_SEG_DIV_MAX = 2;

template <int K, int NT>
static int segs_k(int q, int strips, int batch) {
    if constexpr (kApplyPush) {
        constexpr int NS = push_streams(K, NT);
        return apply3_segments(q, strips, batch, apply4_ctas_wanted_t<K, NT, NS>() * APPLY_SEG_DIV_MAX, K, NS);
    } else {
        constexpr int NS = packed_streams(K, NT);
        return apply3_segments(q, strips, batch, apply3_ctas_wanted_t<K, NT, NS>() * APPLY_SEG_DIV_MAX, K, NS);
    }
}

template <int K>
static int segs_kn(int nt, int q, int strips, int batch) {
    if constexpr (packed_apply_ok(K, 8)) {
        if (nt == 8) return segs_k<K, 8>(q, strips, batch);
    }
    if constexpr (packed_apply_ok(K, 5)) return segs_k<K, 5>(q, strips, batch);
    return 1;
}

// CTAs per instance of the PCG-form apply of (K, nt, precision) at size q and batch: the
// number of per-CTA partials each launch writes.
int apply_pcg_ctas_per_instance(int K, int nt, bool fp64, int q, int batch) {
    const int strips = (q + TB - 1) / TB;
    if (!apply_pcg_packed(K, nt, fp64)) {
        const int TA = apply_pcg_rows_per_cta(K, nt, fp64);
        return strips * ((q + TA - 1) / TA);
    }
    switch (K) {
        case 1: return strips * segs_kn<1>(nt, q, strips, batch);
        case 2: return strips * segs_kn<2>(nt, q, strips, batch);
        case 3: return strips * segs_kn<3>(nt, q, strips, batch);
        default: return strips * segs_kn<4>(nt, q, strips, batch);
    }
}
