// Arithmetic peak probes: the FMA issue rate of this GPU in FP64 and FP32,
// measured with a register-resident loop of independent FMA chains and CUDA
// events.  The FP64 rate bounds the FP64 outer operator apply; both are the
// denominators of the library's ALU roofline reports.  (No counterpart in
// the paper.)
#include "dm_common.cuh"

namespace dm {

namespace {

constexpr int kChains = 8;

// Every thread runs kChains independent chains a <- a * b + c for `iters`
// steps; the results are stored only when flag != 0 (never, in practice) so
// the loop cannot be removed.
template <typename C>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, C b, C c, int flag, C* __restrict__ out) {
    C a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (C)(threadIdx.x + k) * (C)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    C acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k];
    if (flag) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <typename C>
double fma_rate(cudaStream_t s, int blocks, int iters) {
    DBuf<C> out((size_t)blocks * 256, false);
    cudaEvent_t e0, e1;
    note_allocation();
    DM_CUDA(cudaEventCreate(&e0));
    note_allocation();
    DM_CUDA(cudaEventCreate(&e1));
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        DM_CUDA(cudaEventRecord(e0, s));
        launch("k_fma_loop", k_fma_loop<C>, blocks, 256, 0, s, iters, (C)0.999999, (C)1e-7, 0, out.get());
        DM_CUDA(cudaEventRecord(e1, s));
        DM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        DM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms > 0.f)   // the first launch warms up
            best = std::max(best, 2.0 * kChains * (double)iters * blocks * 256 / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

void probe_fma_rates(cudaStream_t s, double* fp64_flops, double* fp32_flops) {
    int dev = 0, sms = 0;
    DM_CUDA(cudaGetDevice(&dev));
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    if (fp64_flops) *fp64_flops = fma_rate<double>(s, blocks, 4096);
    if (fp32_flops) *fp32_flops = fma_rate<float>(s, blocks, 1 << 16);
}

}  // namespace dm
