// fw_probe.cu -- measurement helper, not on the substep path: the L2 read bandwidth of
// the device, for the L2 roofline of kernels whose working set stays in L2 (the SDF
// query reads one grid shared by every environment).
//
// A buffer far smaller than L2 is filled, then read `iters` times by a grid of
// SM-count x 8 blocks with 16-byte loads that bypass L1 (ld.global.cg), so every load
// is served by L2.  Bandwidth = iters x bytes / the CUDA-event time of the reads.
#include "fw_internal.h"

namespace fw {
namespace {

__global__ void probe_fill_kernel(float4 *buf, long long n4) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        buf[i] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
}

__global__ void __launch_bounds__(256) probe_l2_read_kernel(const float4 *__restrict__ buf, long long n4, int iters,
                                                            float *sink) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it) {
        long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        // four independent loads in flight per thread
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc += (a.x + b.y) + (c.z + d.w);
        }
        for (; i < n4; i += stride) acc += __ldcg(buf + i).x;
    }
    if (acc == -1.0f) *sink = acc;   // never true (the buffer holds ones); keeps the loads
}

}  // namespace

cudaError_t measure_l2_read(int device, long long bytes, int iters, float *gbs) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const long long n4 = bytes / 16;
    float4 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s = nullptr;
    e = cudaMalloc(&buf, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        const int grid = n_sm * 8;
        probe_fill_kernel<<<grid, 256, 0, s>>>(buf, n4);
        probe_l2_read_kernel<<<grid, 256, 0, s>>>(buf, n4, 2, sink);   // warm-up: lines into L2
        cudaEventRecord(a, s);
        probe_l2_read_kernel<<<grid, 256, 0, s>>>(buf, n4, iters, sink);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) *gbs = (float)((double)iters * (double)n4 * 16.0 / (ms * 1e-3) / 1e9);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    if (buf) cudaFree(buf);
    return e;
}

}  // namespace fw
