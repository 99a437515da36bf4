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

constexpr int kChunk = 1024;          // input samples per pack CTA and per class_index step
constexpr int kPackRows = 32;         // SNP rows per pack CTA (lane r stores row r)
constexpr int kPackThreads = 256;
constexpr int kUnits = kChunk / 16 + 1;        // 16-byte units of a staged row (with slack)
constexpr int kRowBytes = 16 * kUnits;         // 1040: the chunk from the 16-byte boundary below it
static_assert(kPackThreads * 4 == kChunk, "four samples per thread in the class split");

// One CTA of kChunk threads: counts[0] = N0, counts[1] = N1 and counts[2 + q] = cases among
// the samples before q * kChunk (the pack CTAs' class offsets); flags phenotype values > 1.
__global__ void __launch_bounds__(kChunk)
class_index_kernel(const uint8_t* __restrict__ pheno, int N, int* __restrict__ counts, Ctrl* ctrl) {
    int cases = 0, bad = 0;
    for (int q = 0; q * kChunk < N; ++q) {
        const int s = q * kChunk + (int)threadIdx.x;
        const int v = s < N ? pheno[s] : 0;
        bad |= (v > 1);
        if (threadIdx.x == 0) counts[2 + q] = cases;
        cases += __syncthreads_count(v == 1);
    }
    if (bad) atomicOr(&ctrl->status, kStBadPhenotype);
    if (threadIdx.x == 0) {
        counts[0] = N - cases;
        counts[1] = cases;
    }
}

// nonzero iff a byte of w holds a value above 2
__device__ __forceinline__ uint32_t bad_bytes(uint32_t w) {
    return (w & 0xFCFCFCFCu) | (w & (w >> 1) & 0x01010101u);
}

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// CTA (x, y): input samples [1024 x, 1024 x + 1024) of SNP rows [32 y, 32 y + 32).
//  1. the 32 row segments are staged in shared memory with 16-byte loads (from the 16-byte
//     boundary at or below each segment, so any row stride works);
//  2. the chunk's samples are split by class in input order (block scan of the phenotype),
//     giving each class's local sample offsets; the class positions of the chunk start at
//     counts[2 + x] (cases) and 1024 x - counts[2 + x] (controls);
//  3. per 128-sample group of a class that the chunk touches, a warp forms the words of all
//     32 rows with two ballots per (row, 32 samples) and lane r stores row r's group as one
//     16-byte word per plane (consecutive lanes hold consecutive SNPs: coalesced stores).  A
//     group whose samples all lie in this chunk is stored; a group shared with a neighbouring
//     chunk is OR-ed word by word into the planes, which are zeroed before the launch.
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const uint8_t* __restrict__ geno, const uint8_t* __restrict__ pheno, int M, int N,
            const int* __restrict__ counts, int N0, int N1, Planes pl, uint4* __restrict__ planes,
            Ctrl* ctrl) {
    __shared__ __align__(16) uint8_t tile[kPackRows][kRowBytes];
    __shared__ uint16_t idx[2][kChunk];
    __shared__ int s_shift[kPackRows];
    __shared__ int s_warp[kPackThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int s0 = blockIdx.x * kChunk;
    const int ns = min(kChunk, N - s0);
    const int m0 = blockIdx.y * kPackRows;
    uint32_t bad = 0;

    // 1. stage the row segments [m N + s0, m N + s0 + ns)
    for (int t = tid; t < kPackRows * kUnits; t += kPackThreads) {
        const int r = t / kUnits, u = t - r * kUnits;
        const int m = m0 + r;
        if (m >= M) {  // rows past the data set are never stored; keep their lookups in range
            if (u == 0) s_shift[r] = 0;
            continue;
        }
        const uint8_t* p0 = geno + (size_t)m * N + s0;
        const uintptr_t al = reinterpret_cast<uintptr_t>(p0) & ~static_cast<uintptr_t>(15);
        const int shift = (int)(reinterpret_cast<uintptr_t>(p0) - al);
        if (u == 0) s_shift[r] = shift;
        const int lo = 16 * u - shift;             // first byte of the unit, relative to p0
        if (lo + 16 <= 0 || lo >= ns) continue;    // holds no byte of the segment
        uint4 v;
        if (lo >= 0 && lo + 16 <= ns) {
            v = __ldg(reinterpret_cast<const uint4*>(al) + u);
        } else {  // an end of the segment: only the segment's own bytes are read
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (lo + e >= 0 && lo + e < ns) w[e >> 2] |= (uint32_t)p0[lo + e] << (8 * (e & 3));
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        bad |= bad_bytes(v.x) | bad_bytes(v.y) | bad_bytes(v.z) | bad_bytes(v.w);
        *reinterpret_cast<uint4*>(&tile[r][16 * u]) = v;
    }

    // 2. class split of the chunk: idx[c][local class position] = sample offset in the chunk
    int c1[4], n1 = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int o = 4 * tid + e;
        c1[e] = (o < ns && pheno[s0 + o] == 1) ? 1 : 0;
        n1 += c1[e];
    }
    const int incl = warp_incl_scan(n1);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int before = 0, total1 = 0;
#pragma unroll
    for (int w = 0; w < kPackThreads / 32; ++w) {
        const int v = s_warp[w];
        before += (w < wid) ? v : 0;
        total1 += v;
    }
    int p1 = before + incl - n1;          // cases before this thread's first sample
    int p0 = 4 * tid - p1;                // controls before it
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int o = 4 * tid + e;
        if (o < ns) {
            if (c1[e]) idx[1][p1++] = (uint16_t)o;
            else idx[0][p0++] = (uint16_t)o;
        }
    }
    __syncthreads();

    // 3. groups of 128 class positions touched by this chunk, both classes, spread over warps
    const int a1 = counts[2 + blockIdx.x], a0 = s0 - a1;
    const int nloc[2] = {ns - total1, total1};
    const int acls[2] = {a0, a1};
    const int gl0 = a0 >> 7, gl1 = a1 >> 7;
    const int G0 = nloc[0] ? ((a0 + nloc[0] - 1) >> 7) - gl0 + 1 : 0;
    const int G1 = nloc[1] ? ((a1 + nloc[1] - 1) >> 7) - gl1 + 1 : 0;
    const int m = m0 + lane;
    for (int it = wid; it < G0 + G1; it += kPackThreads / 32) {
        const int c = it < G0 ? 0 : 1;
        const int g = c ? gl1 + (it - G0) : gl0 + it;
        const int a = acls[c], n = nloc[c];
        const int Nc = c ? N1 : N0;
        const bool owned = 128 * g >= a && min(128 * g + 128, Nc) <= a + n;
        uint32_t w0[4], w1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int loc = 128 * g + 32 * q + lane - a;
            const bool valid = loc >= 0 && loc < n;
            const int o = valid ? idx[c][loc] : 0;
            w0[q] = 0u;
            w1[q] = 0u;
#pragma unroll 8
            for (int r = 0; r < kPackRows; ++r) {
                const int gv = valid ? tile[r][s_shift[r] + o] : 3;
                const uint32_t b0 = __ballot_sync(0xffffffffu, gv == 0);
                const uint32_t b1 = __ballot_sync(0xffffffffu, gv == 1);
                if (lane == r) {
                    w0[q] = b0;
                    w1[q] = b1;
                }
            }
        }
        if (m < M) {
            uint4* d0 = planes + pl.coff[c] + (size_t)g * M + m;
            uint4* d1 = planes + pl.coff[c] + (size_t)(pl.W4[c] + g) * M + m;
            if (owned) {
                *d0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *d1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            } else {
                uint32_t* e0 = reinterpret_cast<uint32_t*>(d0);
                uint32_t* e1 = reinterpret_cast<uint32_t*>(d1);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (w0[q]) atomicOr(e0 + q, w0[q]);
                    if (w1[q]) atomicOr(e1 + q, w1[q]);
                }
            }
        }
    }
    if (bad) atomicOr(&ctrl->status, kStBadGenotype);
}

}  // namespace

size_t class_counts_len(int N) { return 2 + (size_t)(N + kChunk - 1) / kChunk; }

cudaError_t launch_class_index(const uint8_t* pheno, int N, int* counts, Ctrl* ctrl,
                               cudaStream_t st) {
    class_index_kernel<<<1, kChunk, 0, st>>>(pheno, N, counts, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* geno, const uint8_t* pheno, int M, int N, const int* counts,
                        int N0, int N1, const Planes& pl, uint4* planes, Ctrl* ctrl, cudaStream_t st) {
    const size_t n4 = 2ull * (pl.W4[0] + pl.W4[1]) * (size_t)M;
    cudaError_t e = cudaMemsetAsync(planes, 0, n4 * sizeof(uint4), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((N + kChunk - 1) / kChunk, (M + kPackRows - 1) / kPackRows);
    pack_kernel<<<grid, kPackThreads, 0, st>>>(geno, pheno, M, N, counts, N0, N1, pl, planes, ctrl);
    return cudaGetLastError();
}

}  // namespace epi3
