// FP32 instantiations of the banded operator apply (mixed-precision inner solve).
#include "apply_impl.cuh"

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

template <int K>
static mofem_status pcg_nt_f32(int nt, const CUtensorMap& mZ, const CUtensorMap& mQ, const ApplyPcgArgs& a, int batch,
                               cudaStream_t st) {
    if (nt == 5) return launch_pcg_t<float, K, 5, false>(mZ, mQ, a, batch, st);
    if (nt == 8) return launch_pcg_t<float, K, 8, false>(mZ, mQ, a, batch, st);
    return MOFEM_ERR_UNSUPPORTED;
}

mofem_status launch_apply_pcg(int K, int nt, bool fp64, const CUtensorMap& mZ, const CUtensorMap& mQ,
                              const ApplyPcgArgs& a, int batch, cudaStream_t st) {
    if (fp64) return launch_apply_pcg_f64(K, nt, mZ, mQ, a, batch, st);
    switch (K) {
        case 1: return pcg_nt_f32<1>(nt, mZ, mQ, a, batch, st);
        case 2: return pcg_nt_f32<2>(nt, mZ, mQ, a, batch, st);
        case 3: return pcg_nt_f32<3>(nt, mZ, mQ, a, batch, st);
        case 4: return pcg_nt_f32<4>(nt, mZ, mQ, a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

int apply_pcg_rows_per_cta(int K) {
    switch (K) {
        case 1: return Geo<1>::TA_T;
        case 2: return Geo<2>::TA_T;
        case 3: return Geo<3>::TA_T;
        default: return Geo<4>::TA_T;
    }
}
