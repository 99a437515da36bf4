// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/epi3.h"

namespace epi3 {

constexpr int kCells = 27;
constexpr int kWordsPerGroup = 4;       // uint4 groups of 32-bit words: 128 samples
constexpr int kSamplesPerGroup = 128;
constexpr int kMaxSamples = 131072;     // popc path: pair planes must fit in shared memory
constexpr int kFinalCap = 8192;         // candidates rescored in FP64 and sorted on one CTA
constexpr int kCtaCand = 1024;          // per-CTA shared candidate buffer (power of two)

// Status bits written by kernels into Ctrl::status.
constexpr int kStBadGenotype = 1;
constexpr int kStBadPhenotype = 2;
constexpr int kStCandOverflow = 4;
constexpr int kStFinalOverflow = 8;
constexpr int kStInternal = 16;
constexpr int kStBadIndex = 32;

// Device control block of one scan.  Zeroed (then thr set to +inf) before each scan.
struct Ctrl {
    unsigned long long work;      // next work item (pair index offset)
    unsigned int thr;             // global FP32 threshold, float bits (non-negative floats)
    unsigned int n_cand;          // global candidate count
    int status;                   // kSt* bits
    unsigned int n_final;         // candidates admitted to FP64 rescoring
    float t_final;                // FP32 threshold of the rescoring stage
    float kth;                    // k-th smallest FP32 score
    unsigned int n_out;           // rows written to the result
    unsigned int pad_[7];
};

struct Cand {                     // one FP32 candidate
    float s;
    int i, j, k;
};

struct Final {                    // one FP64-rescored candidate
    double s;
    unsigned long long key;       // (i << 42) | (j << 21) | k
};

// Bit planes of one data set.  For class c, plane p (0: genotype 0, 1: genotype 1),
// 128-sample group w4 and SNP m, the uint4 at planes[coff[c] + (p * W4[c] + w4) * M + m]
// holds samples 128*w4 .. 128*w4+127 of that class (bit b of word q = sample 32q+b).
// Bits past the class size are 0 in both planes, i.e. they read as genotype 2.
struct Planes {
    const uint4* planes;
    int M;
    int W4[2];
    long long coff[2];
    int pad[2];                   // pad samples per class: 128 * W4[c] - N_c
};

struct K2Tables {
    const float2* lf2;            // lf(n) = hi + lo, hi on a 2^-g grid (exact sums)
    const double* lf64;           // lf(n), same values as the host recurrence
    float rel, abs_;              // |s32 - s64| <= rel * s + abs_
};

struct ScanArgs {
    Planes pl;
    K2Tables k2;
    Ctrl* ctrl;
    Cand* cand;
    long long cand_cap;
    long long pair_begin, pair_end;
    int top_k;
};

// launchers (return cudaError_t of the launch)
cudaError_t launch_class_index(const uint8_t* pheno, int N, int* perm, int* counts, Ctrl* ctrl,
                               cudaStream_t st);
cudaError_t launch_pack(const uint8_t* geno, int M, int N, const int* perm, int N0, int N1,
                        const Planes& pl, uint4* planes, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_scan_popc(const ScanArgs& a, int grid, int block, size_t smem, cudaStream_t st);
size_t scan_popc_smem(const Planes& pl);
cudaError_t scan_popc_occupancy(int block, size_t smem, int* ctas_per_sm);
cudaError_t launch_select(Ctrl* ctrl, const Cand* cand, long long cand_cap, int top_k,
                          float rel, float abs_, cudaStream_t st);
cudaError_t launch_rescore(const Planes& pl, const K2Tables& k2, Ctrl* ctrl, const Cand* cand,
                           long long cand_cap, Final* fin, int grid, cudaStream_t st);
cudaError_t launch_final(Ctrl* ctrl, const Final* fin, int top_k, double* out_scores,
                         int* out_trip, cudaStream_t st);
cudaError_t launch_tables(const Planes& pl, const K2Tables* k2, long long n, const int* trip,
                          int* out_counts, float* out_s32, double* out_s64, Ctrl* ctrl,
                          cudaStream_t st);
cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st);

// Message returned by epi3_last_error() on this thread.
void set_last_error(const char* msg);

// ---------------------------------------------------------------- device helpers

// Upper end of the FP32 band that can still hold the answer, given the k-th best
// FP32 score: every triplet of the true top-k has s32 <= kth*(1+4 rel) + 4 abs.
__host__ __device__ inline float band_threshold(float kth, float rel, float abs_) {
#ifdef __CUDA_ARCH__
    return __fmaf_ru(kth, 1.0f + 4.0f * rel, 4.0f * abs_);
#else
    return kth * (1.0f + 4.0f * rel) + 4.0f * abs_;
#endif
}

__host__ __device__ inline unsigned long long pack_key(int i, int j, int k) {
    return ((unsigned long long)i << 42) | ((unsigned long long)j << 21) | (unsigned long long)k;
}

// Pair index p in the order (j ascending, then i ascending): p = j(j-1)/2 + i.
__device__ inline void decode_pair(long long p, int* i, int* j) {
    long long jj = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)p)) * 0.5);
    while (jj * (jj - 1) / 2 > p) --jj;
    while ((jj + 1) * jj / 2 <= p) ++jj;
    *j = (int)jj;
    *i = (int)(p - jj * (jj - 1) / 2);
}

// FP32 K2 (Eq. 1) of a 2 x 27 table.  hi parts are multiples of 2^-g below 2^(24-g):
// every hi difference and partial sum is exact, so only the lo parts and the final
// add round.
__device__ __forceinline__ float k2_f32(const int* r0, const int* r1, const float2* lf2) {
    float ah = 0.f, al = 0.f;
#pragma unroll
    for (int c = 0; c < kCells; ++c) {
        const float2 a = __ldg(lf2 + r0[c] + r1[c] + 1);
        const float2 b = __ldg(lf2 + r0[c]);
        const float2 d = __ldg(lf2 + r1[c]);
        ah += __fsub_rn(__fsub_rn(a.x, b.x), d.x);
        al += __fsub_rn(__fsub_rn(a.y, b.y), d.y);
    }
    return __fadd_rn(ah, al);
}

// FP64 K2 (Eq. 1) in cell order 0..26: term = (lf[r+1] - lf[r0]) - lf[r1], sum from 0.0.
__device__ inline double k2_f64(const int* r0, const int* r1, const double* lf64) {
    double s = 0.0;
    for (int c = 0; c < kCells; ++c) {
        const double t = __dsub_rn(__dsub_rn(lf64[r0[c] + r1[c] + 1], lf64[r0[c]]), lf64[r1[c]]);
        s = __dadd_rn(s, t);
    }
    return s;
}

}  // namespace epi3
