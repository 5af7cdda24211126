// mofem_precond_noalloc: the BF16 tensor-core preconditioner Z = P^{-1}(R)
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they apply the
// preconditioner: code that must not trigger the implicit device-wide
// synchronisation of cudaMalloc/cudaFree in a latency-critical loop, or code
// running under a memory budget owned by its own allocator.  The regular
// mofem_precond(MOFEM_MIXED_BF16) allocates its BF16 operand copies and GEMM
// intermediates on first use; this variant keeps them in a file-scope static
// device array instead, so a call allocates nothing.
//
// The array holds 8 BF16 matrices of at most MOFEM_NOALLOC_MAX_ELEMS elements
// each (4 MiB in total) and is held by every GPU that loads the library until
// the process exits.  Every call shares it and it keeps the last call's
// contents: calls that overlap on the GPU (different streams, or different
// handles on the same device) race on it and must be serialised by the caller.
// Nothing in it has to start at zero: the tensor-core loads only read within
// the q x q extent (out-of-range rows and columns are filled with zeros by the
// copy engine) and every GEMM overwrites its output before the next one reads it.
#include "internal.h"

#include <cuda_bf16.h>
#include <cstdio>

#define MOFEM_NOALLOC_MAX_ELEMS (1 << 18)   // batch * q * ld per matrix, e.g. one instance with q <= 512

static __device__ __align__(256) __nv_bfloat16 g_noalloc_scratch[8 * (size_t)MOFEM_NOALLOC_MAX_ELEMS];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

// dst[r][c] = bf16(src[c][r]) (transpose = 1) or bf16(src[r][c]); n x n, leading dimensions given.
// Rounded through FP32, as the handle's own BF16 operand copies are, so both entry points
// multiply by the same operands.
__global__ void k_f64_to_bf16(const double* src, long long s_bs, int s_ld, __nv_bfloat16* dst, long long d_bs,
                              int d_ld, int n, int transpose) {
    __shared__ double tile[32][33];
    const int inst = blockIdx.z;
    src += (size_t)inst * s_bs;
    dst += (size_t)inst * d_bs;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int y = by + j, x = bx + threadIdx.x;
        tile[j][threadIdx.x] = (x < n && y < n) ? src[(size_t)y * s_ld + x] : 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        if (transpose) {
            const int y = bx + j, x = by + threadIdx.x;   // dst row = src column
            if (x < n && y < n) dst[(size_t)y * d_ld + x] = __float2bfloat16_rn((float)tile[threadIdx.x][j]);
        } else {
            const int y = by + j, x = bx + threadIdx.x;
            if (x < n && y < n) dst[(size_t)y * d_ld + x] = __float2bfloat16_rn((float)tile[j][threadIdx.x]);
        }
    }
}

}  // namespace

extern "C" mofem_status mofem_precond_noalloc(mofem_handle h, const float* R, float* Z, int ld, cudaStream_t stream) {
    if (!h || !R || !Z || ld < h->q) return MOFEM_ERR_INVALID_ARG;
    const int q = h->q, lds = h->ld, B = h->batch;
    const long long per = (long long)q * lds;
    if (per * B > MOFEM_NOALLOC_MAX_ELEMS) {
        char buf[160];
        snprintf(buf, sizeof buf, "mofem_precond_noalloc: batch*q*ld = %lld exceeds the static scratch limit %d",
                 per * B, MOFEM_NOALLOC_MAX_ELEMS);
        mofem_set_last_error(buf, __FILE__, __LINE__);
        return MOFEM_ERR_INVALID_ARG;
    }
    // Device address of the static array, looked up once per device with that
    // device current (the host-side symbol is only a stand-in, not a device address).
    // Under lazy module loading this first lookup may load the module, which is when
    // the array itself is allocated.
    int dev = 0;
    MOFEM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MOFEM_ERR_UNSUPPORTED;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        MOFEM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    __nv_bfloat16* base = static_cast<__nv_bfloat16*>(g_scratch_addr[dev]);
    TcBuffers b;
    b.ld = lds;
    void** slots[8] = {&b.Q1, &b.Q1T, &b.Q2, &b.Q2T, &b.Rop, &b.X1T, &b.WT, &b.Y};
    for (int i = 0; i < 8; ++i) *slots[i] = base + (size_t)i * MOFEM_NOALLOC_MAX_ELEMS;
    // BF16 operand copies of the FP64 eigenvector matrices (owned by the handle) and of R
    dim3 tg((q + 31) / 32, (q + 31) / 32, B), tb(32, 8);
    k_f64_to_bf16<<<tg, tb, 0, stream>>>(h->Q1_64, per, lds, (__nv_bfloat16*)b.Q1, per, lds, q, 0);
    k_f64_to_bf16<<<tg, tb, 0, stream>>>(h->Q1_64, per, lds, (__nv_bfloat16*)b.Q1T, per, lds, q, 1);
    dim3 tg1((q + 31) / 32, (q + 31) / 32, 1);
    k_f64_to_bf16<<<tg1, tb, 0, stream>>>(h->Q2_64, per, lds, (__nv_bfloat16*)b.Q2, per, lds, q, 0);
    k_f64_to_bf16<<<tg1, tb, 0, stream>>>(h->Q2_64, per, lds, (__nv_bfloat16*)b.Q2T, per, lds, q, 1);
    MOFEM_CUDA_TRY(cudaGetLastError());
    MOFEM_TRY(launch_convert(R, 0, (long long)ld * q, ld, b.Rop, 2, per, lds, q, q, B, stream));
    return tc_precond_buffers(h, b, Z, ld, (long long)ld * q, stream);
}
