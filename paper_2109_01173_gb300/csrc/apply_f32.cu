// FP32 instantiations of the banded operator apply (mixed-precision inner solve).
#include "apply_impl.cuh"

using namespace mofem_apply_impl;

mofem_status launch_apply_f64(int K, int nt, int mode, const ApplyArgs& a, int batch, cudaStream_t st);

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
        case 1: return Geo<1>::TA;
        case 2: return Geo<2>::TA;
        case 3: return Geo<3>::TA;
        default: return Geo<4>::TA;
    }
}
