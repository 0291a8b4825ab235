// FP32 FMA throughput probe: the measured denominator of the ALU roofline of the
// spreading and gather kernels, which are bound by FP32 fused multiply-adds.
//
// Every thread runs kChains independent FMA chains x <- x * m + c for `iters` rounds,
// enough independent work per warp to cover the FMA latency at 8 warps per scheduler,
// so the launch runs at the FP32 pipe's issue rate.  The caller times the launch with
// CUDA events on `stream`; flop = 2 * chains * iters * threads.
#include "se_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, float m, float c, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // the store depends on every chain, so none of them is dead code; m and c keep the
    // values bounded (|m| < 1), and a NaN never arises from finite inputs
    if (s == 12345.678f) sink[0] = s;
}

}  // namespace

extern "C" int se_fp32_fma_probe(int device, void *stream, int iters, float *sink, double *flop, int *sms)
{
    if (iters < 1 || !sink || !flop) return SE_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SE_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SE_ERR_CUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || nsm < 1) {
        cudaSetDevice(prev);
        return SE_ERR_CUDA;
    }
    const int blocks = nsm * kBlocksPerSm;
    cudaGetLastError();
    fma_probe_kernel<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(iters, 0.999999f, 1e-7f, sink);
    const cudaError_t e = cudaGetLastError();
    cudaSetDevice(prev);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    *flop = 2.0 * kChains * (double)iters * blocks * kThreads;
    if (sms) *sms = nsm;
    return SE_OK;
}
