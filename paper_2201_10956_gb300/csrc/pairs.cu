// Pair tables and single-SNP marginals for the 8-cell counting forms.
//
// For SNPs m1 < m2 and class c: the 2 x 2 counts of genotypes {0,1} x {0,1} (the pairwise
// frequency table of Sec. III restricted to genotypes 0 and 1), from the bit planes with
// AND + POPC.  Together with the marginals they turn the 8 directly counted cells of a
// triplet (every genotype in {0,1}) into all 27 (derive27).  Bits past a class's size are 0
// in both planes, so they never reach these counts.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

constexpr int kPairThreads = 128;

__global__ void __launch_bounds__(kPairThreads)
pair_tables_kernel(Planes pl, int4* __restrict__ pt, int2* __restrict__ marg, long long n_pairs) {
    const int m2 = blockIdx.x * kPairThreads + threadIdx.x;
    const int M = pl.M;
    if (m2 >= M) return;
    for (int m1 = blockIdx.y; m1 < M; m1 += gridDim.y) {
    const bool pair = m2 > m1;
    const bool single = (m1 == 0);  // one row of blocks also writes the marginals of m2
    if (!pair && !single) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int W4 = pl.W4[c];
        const uint4* base = pl.planes + pl.coff[c];
        const size_t ps = (size_t)W4 * M;
        int n00 = 0, n01 = 0, n10 = 0, n11 = 0, m0 = 0, mo = 0;
        for (int w4 = 0; w4 < W4; ++w4) {
            const size_t o = (size_t)w4 * M;
            const uint4 y0 = __ldg(base + o + m2), y1 = __ldg(base + ps + o + m2);
            if (pair) {
                const uint4 x0 = __ldg(base + o + m1), x1 = __ldg(base + ps + o + m1);
                n00 += __popc(x0.x & y0.x) + __popc(x0.y & y0.y) + __popc(x0.z & y0.z) + __popc(x0.w & y0.w);
                n01 += __popc(x0.x & y1.x) + __popc(x0.y & y1.y) + __popc(x0.z & y1.z) + __popc(x0.w & y1.w);
                n10 += __popc(x1.x & y0.x) + __popc(x1.y & y0.y) + __popc(x1.z & y0.z) + __popc(x1.w & y0.w);
                n11 += __popc(x1.x & y1.x) + __popc(x1.y & y1.y) + __popc(x1.z & y1.z) + __popc(x1.w & y1.w);
            }
            if (single) {
                m0 += __popc(y0.x) + __popc(y0.y) + __popc(y0.z) + __popc(y0.w);
                mo += __popc(y1.x) + __popc(y1.y) + __popc(y1.z) + __popc(y1.w);
            }
        }
        if (pair) pt[c * n_pairs + pair_index(m1, m2)] = make_int4(n00, n01, n10, n11);
        if (single) marg[(size_t)c * M + m2] = make_int2(m0, mo);
    }
    }
}

__global__ void pair_floats_kernel(const int4* __restrict__ pt, const int2* __restrict__ marg,
                                   long long n_pt, long long n_marg, float4* __restrict__ ptf,
                                   float2* __restrict__ margf) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_pt + n_marg;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < n_pt) {
            const int4 q = pt[t];
            ptf[t] = make_float4((float)(q.x + 3), (float)(q.y + 3), (float)(q.z + 3), (float)(q.w + 3));
        } else {
            const int2 q = marg[t - n_pt];
            margf[t - n_pt] = make_float2((float)(q.x + 9), (float)(q.y + 9));
        }
    }
}

}  // namespace

cudaError_t launch_pair_floats(const int4* pt, const int2* marg, long long n_pairs, int M,
                               float4* ptf, float2* margf, cudaStream_t st) {
    const long long n = 2 * n_pairs + 2LL * M;
    const int blocks = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    pair_floats_kernel<<<blocks, 256, 0, st>>>(pt, marg, 2 * n_pairs, 2LL * M, ptf, margf);
    return cudaGetLastError();
}

cudaError_t launch_pair_tables(const Planes& pl, int4* pt, int2* marg, long long n_pairs,
                               cudaStream_t st) {
    dim3 grid((pl.M + kPairThreads - 1) / kPairThreads, pl.M < 65535 ? pl.M : 65535);
    pair_tables_kernel<<<grid, kPairThreads, 0, st>>>(pl, pt, marg, n_pairs);
    return cudaGetLastError();
}

}  // namespace epi3
