// Throughput of lg2.approx.ftz.f32, the instruction the tensor scans' table-free K2 bound spends
// 81 times per triplet (three per cell, 27 cells): eight independent chains per thread, 4 CTAs of
// 8 warps per SM, issued back to back.  Prints lg2 results per SM per clock, the peak behind the
// epilogue's roofline.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kWarps = 8;   // per CTA
constexpr int kChains = 8;  // independent lg2 chains per thread

__global__ void __launch_bounds__(32 * kWarps) lg2_kernel(int iters, unsigned long long* cycles,
                                                           float* sink) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1.5f + 0.001f * (float)(threadIdx.x + 37 * j);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            float y;
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
            x[j] = y + 2.0f;   // stays in [2, 3): the next lg2 depends on this one
        }
    }
    const long long t1 = clock64();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(cycles, (unsigned long long)(t1 - t0));
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == 12345.f) sink[0] = s;
}

int main() {
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    unsigned long long* cyc = nullptr;
    float* sink = nullptr;
    cudaMalloc(&cyc, sizeof(unsigned long long));
    cudaMalloc(&sink, sizeof(float));
    const int ctas_per_sm = 4, grid = sms * ctas_per_sm, iters = 4096;
    lg2_kernel<<<grid, 32 * kWarps>>>(64, cyc, sink);  // warm-up
    cudaMemset(cyc, 0, sizeof(unsigned long long));
    lg2_kernel<<<grid, 32 * kWarps>>>(iters, cyc, sink);
    const cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h = 0;
    cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
    const double cyc_cta = (double)h / grid;   // the CTAs of one SM run concurrently
    const double lg2_per_sm = (double)ctas_per_sm * kWarps * 32 * kChains * iters;
    printf("SMs %d, clock %d MHz\n", sms, clk_khz / 1000);
    printf("lg2.approx.ftz.f32: %s, %.1f cycles per CTA, %.2f lg2/SM/clk\n", cudaGetErrorString(e),
           cyc_cta, lg2_per_sm / cyc_cta);
    cudaFree(cyc);
    cudaFree(sink);
    return e == cudaSuccess ? 0 : 1;
}
