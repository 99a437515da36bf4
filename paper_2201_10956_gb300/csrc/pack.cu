// Class split and bit-plane packing (Sec. III Fig. 1 binarisation, Sec. IV-A data split).
//
// The samples are split into controls (class 0) and cases (class 1), keeping their
// input order inside each class.  For every SNP and class two bit planes are stored:
// genotype 0 and genotype 1.  The genotype-2 plane is never stored; consumers derive
// it as NOR of the two (Sec. IV-A).  Bits beyond a class's sample count are 0 in both
// planes, so they read as genotype 2 and land in cell (2,2,2) only.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

constexpr int kIndexThreads = 1024;
constexpr int kPackRows = 8;          // SNP rows per pack CTA (one lane per row writes)
constexpr int kPackThreads = 256;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// One CTA: counts the cases, then writes perm[0..N0) = control sample indices and
// perm[N0..N) = case sample indices, both in input order.  counts = {N0, N1}.
__global__ void __launch_bounds__(kIndexThreads)
class_index_kernel(const uint8_t* __restrict__ pheno, int N, int* __restrict__ perm,
                   int* __restrict__ counts, Ctrl* ctrl) {
    __shared__ int s_warp[kIndexThreads / 32];
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int bad = 0, ncase = 0;
    for (int s = tid; s < N; s += kIndexThreads) {
        const int v = pheno[s];
        bad |= (v > 1);
        ncase += (v == 1);
    }
    // block sum of ncase
    for (int d = 16; d > 0; d >>= 1) ncase += __shfl_xor_sync(0xffffffffu, ncase, d);
    if (lane == 0) s_warp[wid] = ncase;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int w = 0; w < kIndexThreads / 32; ++w) t += s_warp[w];
        s_total = t;
    }
    if (bad) atomicOr(&ctrl->status, kStBadPhenotype);
    __syncthreads();
    const int N1 = s_total, N0 = N - N1;
    int cases_before = 0;  // cases in earlier chunks
    for (int base = 0; base < N; base += kIndexThreads) {
        const int s = base + tid;
        const int is_case = (s < N && pheno[s] == 1) ? 1 : 0;
        const int incl = warp_incl_scan(is_case);
        __syncthreads();
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        int warp_off = 0, chunk_total = 0;
        for (int w = 0; w < kIndexThreads / 32; ++w) {
            const int c = s_warp[w];
            if (w < wid) warp_off += c;
            chunk_total += c;
        }
        if (s < N) {
            const int pos1 = cases_before + warp_off + incl - is_case;  // cases before s
            if (is_case) perm[N0 + pos1] = s;
            else perm[s - pos1] = s;
        }
        cases_before += chunk_total;
    }
    if (tid == 0) {
        counts[0] = N0;
        counts[1] = N1;
    }
}

// kPackRows SNP rows per CTA.  Each warp builds 32-sample words: lane l reads the
// genotype of class position 32 w + l, two ballots give the genotype-0 and genotype-1
// words, and lane r keeps row r's pair of words for the store.
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const uint8_t* __restrict__ geno, int M, int N, const int* __restrict__ perm,
            int N0, int N1, Planes pl, uint4* __restrict__ planes, Ctrl* ctrl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int m0 = blockIdx.x * kPackRows;
    const int words0 = 4 * pl.W4[0];
    const int words = words0 + 4 * pl.W4[1];
    int bad = 0;
    for (int q = wid; q < words; q += kPackThreads / 32) {
        const int c = (q < words0) ? 0 : 1;
        const int w = (c == 0) ? q : q - words0;
        const int Nc = (c == 0) ? N0 : N1;
        const int pos = 32 * w + lane;
        const bool valid = pos < Nc;
        const int s = valid ? perm[c * N0 + pos] : 0;
        unsigned my0 = 0u, my1 = 0u;
#pragma unroll
        for (int r = 0; r < kPackRows; ++r) {
            const int m = m0 + r;
            int g = 3;  // pad / absent row: neither plane
            if (valid && m < M) {
                g = geno[(size_t)m * N + s];
                bad |= (g > 2);
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, g == 0);
            const unsigned b1 = __ballot_sync(0xffffffffu, g == 1);
            if (lane == r) {
                my0 = b0;
                my1 = b1;
            }
        }
        const int m = m0 + lane;
        if (lane < kPackRows && m < M) {
            const size_t g4 = (size_t)pl.coff[c] + (size_t)(w >> 2) * M + m;
            uint32_t* p0 = reinterpret_cast<uint32_t*>(planes + g4) + (w & 3);
            uint32_t* p1 = reinterpret_cast<uint32_t*>(planes + g4 + (size_t)pl.W4[c] * M) + (w & 3);
            *p0 = my0;
            *p1 = my1;
        }
    }
    if (bad) atomicOr(&ctrl->status, kStBadGenotype);
}

}  // namespace

cudaError_t launch_class_index(const uint8_t* pheno, int N, int* perm, int* counts, Ctrl* ctrl,
                               cudaStream_t st) {
    class_index_kernel<<<1, kIndexThreads, 0, st>>>(pheno, N, perm, counts, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* geno, int M, int N, const int* perm, int N0, int N1,
                        const Planes& pl, uint4* planes, Ctrl* ctrl, cudaStream_t st) {
    const int grid = (M + kPackRows - 1) / kPackRows;
    pack_kernel<<<grid, kPackThreads, 0, st>>>(geno, M, N, perm, N0, N1, pl, planes, ctrl);
    return cudaGetLastError();
}

}  // namespace epi3
