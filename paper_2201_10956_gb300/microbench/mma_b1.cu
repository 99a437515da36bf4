// Binary tensor-core rate: mma.sync m16n8k256 b1 x b1 -> s32 with AND + POPC (the only 1-bit
// tensor operation on sm_103a; tcgen05 has no 1-bit kind), issued back to back from every warp
// with four independent accumulators.  Prints the bit-MACs per SM per clock (16 x 8 x 256 per
// instruction) and, for reference, the 32-bit AND + POPC rate of the CUDA cores in the same
// shape of loop (32 bit-ops per POPC).
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kWarps = 8;   // per CTA
constexpr int kAcc = 4;     // independent accumulators per warp

__global__ void __launch_bounds__(32 * kWarps) b1_kernel(int iters, unsigned long long* cycles,
                                                          int* sink) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = 0x9E3779B9u * (threadIdx.x + 7 * t + 1);
    b[0] = 0x85EBCA6Bu * (threadIdx.x + 3);
    b[1] = 0xC2B2AE35u * (threadIdx.x + 5);
    int c[kAcc][4];
#pragma unroll
    for (int j = 0; j < kAcc; ++j)
#pragma unroll
        for (int t = 0; t < 4; ++t) c[j][t] = 0;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kAcc; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc "
                "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    const long long t1 = clock64();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(cycles, (unsigned long long)(t1 - t0));
    int s = 0;
#pragma unroll
    for (int j = 0; j < kAcc; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
    if (s == 0x7FFFFFFF) atomicAdd(sink, s);
}

// CUDA-core reference: per 32-bit word, one AND and one POPC, 8 independent chains per thread.
__global__ void __launch_bounds__(32 * kWarps) popc_kernel(int iters, unsigned long long* cycles,
                                                            int* sink) {
    uint32_t x[8], y = 0x85EBCA6Bu * (threadIdx.x + 3);
    int acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        x[j] = 0x9E3779B9u * (threadIdx.x + 7 * j + 1);
        acc[j] = 0;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            acc[j] += __popc(x[j] & y);
            x[j] = x[j] * 0x01000193u + (uint32_t)it;  // keep the words changing
        }
    }
    const long long t1 = clock64();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(cycles, (unsigned long long)(t1 - t0));
    int s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += acc[j];
    if (s == 0x7FFFFFFF) atomicAdd(sink, s);
}

int main() {
    int sms = 0, clk_khz = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    unsigned long long* cyc = nullptr;
    int* sink = nullptr;
    cudaMalloc(&cyc, sizeof(unsigned long long));
    cudaMalloc(&sink, sizeof(int));
    const int ctas_per_sm = 4, grid = sms * ctas_per_sm, iters = 4096;
    // b1 MMA
    b1_kernel<<<grid, 32 * kWarps>>>(64, cyc, sink);  // warm-up
    cudaMemset(cyc, 0, sizeof(unsigned long long));
    b1_kernel<<<grid, 32 * kWarps>>>(iters, cyc, sink);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h = 0;
    cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
    // cycles per CTA; the CTAs of one SM run concurrently
    const double cyc_cta = (double)h / grid;
    const double mma_per_sm = (double)ctas_per_sm * kWarps * kAcc * iters;
    const double bitmac_sm_clk = mma_per_sm * 16.0 * 8.0 * 256.0 / cyc_cta;
    printf("SMs %d, clock %d MHz\n", sms, clk_khz / 1000);
    printf("b1 mma.sync m16n8k256 and.popc: %s, %.1f cycles per CTA, %.1f bit-MAC/SM/clk, "
           "%.2f cycles per warp-instruction per SM\n",
           cudaGetErrorString(e), cyc_cta, bitmac_sm_clk, cyc_cta / (mma_per_sm / 1.0));
    // CUDA-core AND + POPC
    popc_kernel<<<grid, 32 * kWarps>>>(64, cyc, sink);
    cudaMemset(cyc, 0, sizeof(unsigned long long));
    popc_kernel<<<grid, 32 * kWarps>>>(iters, cyc, sink);
    e = cudaDeviceSynchronize();
    cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
    const double cyc_cta2 = (double)h / grid;
    const double popc_per_sm = (double)ctas_per_sm * kWarps * 32 * 8 * iters;
    printf("CUDA-core AND + POPC: %s, %.1f POPC/SM/clk, %.1f bit-op/SM/clk\n", cudaGetErrorString(e),
           popc_per_sm / cyc_cta2, 32.0 * popc_per_sm / cyc_cta2);
    cudaFree(cyc);
    cudaFree(sink);
    return e == cudaSuccess ? 0 : 1;
}
