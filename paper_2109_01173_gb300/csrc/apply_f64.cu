// FP64 instantiations of the banded operator apply: the FP64 form of MO-PCG,
// the FP64 true residual of iterative refinement, and the right-hand side
// (one mass term with index offset).  FP64 runs at a small fraction of the FP32
// rate on this GPU, so the T coefficients are kept in shared memory rather than
// registers to bound register pressure.
#include "apply_impl.cuh"

using namespace mofem_apply_impl;

template <int K, int NT>
static mofem_status dispatch_mode_f64(int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    switch (mode) {
        case APPLY_PLAIN: return launch_t<double, K, NT, APPLY_PLAIN, true>(a, batch, st);
        case APPLY_QUPDATE: return launch_t<double, K, NT, APPLY_QUPDATE, true>(a, batch, st);
        case APPLY_RESIDUAL: return launch_t<double, K, NT, APPLY_RESIDUAL, true>(a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

template <int K>
static mofem_status dispatch_nt_f64(int nt, int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    if (nt == 1) {
        if (mode != APPLY_PLAIN) return MOFEM_ERR_UNSUPPORTED;
        return launch_t<double, K, 1, APPLY_PLAIN, true>(a, batch, st);
    }
    if (nt == 5) return dispatch_mode_f64<K, 5>(mode, a, batch, st);
    if (nt == 8) return dispatch_mode_f64<K, 8>(mode, a, batch, st);
    return MOFEM_ERR_UNSUPPORTED;
}

mofem_status launch_apply_f64(int K, int nt, int mode, const ApplyArgs& a, int batch, cudaStream_t st) {
    switch (K) {
        case 1: return dispatch_nt_f64<1>(nt, mode, a, batch, st);
        case 2: return dispatch_nt_f64<2>(nt, mode, a, batch, st);
        case 3: return dispatch_nt_f64<3>(nt, mode, a, batch, st);
        case 4: return dispatch_nt_f64<4>(nt, mode, a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}

template <int K>
static mofem_status pcg_nt_f64(int nt, const CUtensorMap& mZ, const CUtensorMap& mQ, const ApplyPcgArgs& a, int batch,
                               cudaStream_t st) {
    if (nt == 5) return launch_pcg_t<double, K, 5, true>(mZ, mQ, a, batch, st);
    if (nt == 8) return launch_pcg_t<double, K, 8, true>(mZ, mQ, a, batch, st);
    return MOFEM_ERR_UNSUPPORTED;
}

mofem_status launch_apply_pcg_f64(int K, int nt, const CUtensorMap& mZ, const CUtensorMap& mQ, const ApplyPcgArgs& a,
                                  int batch, cudaStream_t st) {
    switch (K) {
        case 1: return pcg_nt_f64<1>(nt, mZ, mQ, a, batch, st);
        case 2: return pcg_nt_f64<2>(nt, mZ, mQ, a, batch, st);
        case 3: return pcg_nt_f64<3>(nt, mZ, mQ, a, batch, st);
        case 4: return pcg_nt_f64<4>(nt, mZ, mQ, a, batch, st);
        default: return MOFEM_ERR_UNSUPPORTED;
    }
}
