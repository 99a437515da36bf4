// Issue cost of tcgen05.mma kind::mxf4 with both operands in shared memory (M = 128, N = 64 and
// 128, K = 64 FP4 per instruction), three ways: (0) issued by one lane inside a divergent branch,
// (1) by a whole warp with elect.sync inside the asm, (2) as (1) with every operand broadcast from
// lane 0 so that the compiler can prove it warp-uniform.  Descriptors change per MMA like a ring
// of three slots.  One CTA per SM; prints cycles per MMA and the ideal (N / 2 at the dense FP4
// rate).  The shared-memory operand read (A 4 KB + B N x 32 B per MMA) at 128 B/clk bounds N = 64
// at 48 cycles.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool mbar_try(uint32_t a, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
__device__ bool mbar_wait(uint32_t a, unsigned parity) {
    const long long t0 = clock64();
    for (unsigned it = 0;; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 63u) == 0u && clock64() - t0 > 4000000000LL) return false;
    }
}
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
template <int N>
__host__ __device__ constexpr uint32_t idesc_mx() {
    return (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((128u >> 4) << 24);
}
constexpr uint32_t kSf = 448;
constexpr int kSlotBytes = 16384 + 16384;   // A 16 KB + B up to 16 KB

__device__ __forceinline__ void mma_one(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc,
                                        uint32_t sf) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(sf), "r"(sf + 32) : "memory");
}
__device__ __forceinline__ void mma_elect(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc,
                                          uint32_t sf) {
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(sf), "r"(sf + 32) : "memory");
}
__device__ __forceinline__ void commit_elect(uint32_t bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
        ::"r"(bar) : "memory");
}

template <int N, int kStyle>
__global__ void __launch_bounds__(128, 1) mb_kernel(int iters, unsigned long long* out, int* err) {
    extern __shared__ uint8_t raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 3 * kSlotBytes);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < 3 * kSlotBytes / 16; t += blockDim.x)
        reinterpret_cast<uint4*>(base)[t] = make_uint4(0x00220022u, 0x20000000u, 0, 0x00000202u);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    {
        const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
        uint32_t v = 0x7F7F7F7Fu;
        for (int c = 0; c < 64; c += 8)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};"
                         ::"r"(tmem + lane_off + kSf + c), "r"(v) : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t b0 = smem_u32(base);
    const uint32_t idesc = idesc_mx<N>();
    if (kStyle == 0 && threadIdx.x == 0) {
        const long long t0 = clock64();
        int s = 0;
        for (int it = 0; it < iters; ++it) {
            const uint64_t da = sw128_desc(b0 + s * kSlotBytes), db = sw128_desc(b0 + s * kSlotBytes + 16384);
            const uint32_t d = tmem + (uint32_t)((it >> 3) & 1) * 128u;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_one(d, da + 2 * kk, db + 2 * kk, idesc, (it | kk) ? 1u : 0u, tmem + kSf);
            if (++s == 3) s = 0;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(bar)) : "memory");
        if (!mbar_wait(smem_u32(bar), 0)) atomicOr(err, 1);
        atomicAdd(out, (unsigned long long)(clock64() - t0));
    } else if (kStyle > 0 && warp == 0) {
        const long long t0 = clock64();
        int s = 0;
        for (int it = 0; it < iters; ++it) {
            uint32_t pa = b0 + s * kSlotBytes;
            uint32_t d = tmem + (uint32_t)((it >> 3) & 1) * 128u;
            if (kStyle == 2) {
                pa = __shfl_sync(0xffffffffu, pa, 0);
                d = __shfl_sync(0xffffffffu, d, 0);
            }
            const uint64_t da = sw128_desc(pa), db = sw128_desc(pa + 16384);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma_elect(d, da + 2 * kk, db + 2 * kk, idesc, (it | kk) ? 1u : 0u, tmem + kSf);
            if (++s == 3) s = 0;
        }
        commit_elect(smem_u32(bar));
        if (!mbar_wait(smem_u32(bar), 0)) atomicOr(err, 1);
        if (lane == 0) atomicAdd(out, (unsigned long long)(clock64() - t0));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int N, int kStyle>
void run(const char* name, int sms) {
    unsigned long long* out;
    int* err;
    cudaMalloc(&out, 8);
    cudaMalloc(&err, 4);
    cudaMemset(out, 0, 8);
    cudaMemset(err, 0, 4);
    const int smem = 1024 + 3 * kSlotBytes + 64;
    cudaFuncSetAttribute(mb_kernel<N, kStyle>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int iters = 4096;
    mb_kernel<N, kStyle><<<sms, 128, smem>>>(64, out, err);
    cudaError_t e = cudaDeviceSynchronize();
    cudaMemset(out, 0, 8);
    if (e == cudaSuccess) {
        mb_kernel<N, kStyle><<<sms, 128, smem>>>(iters, out, err);
        e = cudaDeviceSynchronize();
    }
    unsigned long long h = 0;
    int herr = 0;
    cudaMemcpy(&h, out, 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    printf("%-34s N=%3d  %s err=%d  %6.1f cycles per MMA (ideal %d)\n", name, N, cudaGetErrorString(e), herr,
           (double)h / sms / iters / 4, N / 2);
    cudaFree(out);
    cudaFree(err);
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    printf("SMs %d\n", sms);
    run<64, 0>("one lane, divergent branch", sms);
    run<64, 1>("whole warp, elect.sync in asm", sms);
    run<64, 2>("whole warp, elect + shfl operands", sms);
    run<128, 0>("one lane, divergent branch", sms);
    run<128, 1>("whole warp, elect.sync in asm", sms);
    run<128, 2>("whole warp, elect + shfl operands", sms);
    return 0;
}
