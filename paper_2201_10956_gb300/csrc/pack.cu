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
constexpr int kPadCol = kChunk;               // 16 bytes of genotype value 3 after each staged row
constexpr int kRowBytes = kChunk + 16;
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
//  1. the 32 row segments are staged in shared memory (16-byte loads where a segment starts on
//     a 16-byte boundary, byte loads otherwise), each row followed by 16 bytes of value 3 that
//     lanes past the class read, so the inner loop needs no bounds test;
//  2. the chunk's samples are split by class in input order (block scan of the phenotype),
//     giving each class's local sample offsets; the class positions of the chunk start at
//     counts[2 + x] (cases) and 1024 x - counts[2 + x] (controls);
//  3. per 32-sample word of a class that the chunk touches, a warp forms the words of all 32
//     rows with one shared-memory byte load and two ballots per row (about 3.5 instructions
//     per output word) and lane r stores row r's word of both planes (consecutive lanes hold
//     consecutive SNPs).  A word whose samples all lie in this chunk is stored; a word shared
//     with a neighbouring chunk is OR-ed into the planes, which are zeroed before the launch.
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const uint8_t* __restrict__ geno, const uint8_t* __restrict__ pheno, int M, int N,
            const int* __restrict__ counts, int N0, int N1, Planes pl, uint4* __restrict__ planes,
            Ctrl* ctrl) {
    __shared__ __align__(16) uint8_t tile[kPackRows][kRowBytes];
    __shared__ uint16_t idx[2][kChunk];
    __shared__ int s_warp[kPackThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int s0 = blockIdx.x * kChunk;
    const int ns = min(kChunk, N - s0);
    const int m0 = blockIdx.y * kPackRows;
    uint32_t bad = 0;

    // 1. stage the row segments [m N + s0, m N + s0 + ns) at tile[r][0 .. ns).  Rows whose
    //    segment starts on a 16-byte boundary move in 16-byte units, every thread issuing all of
    //    its loads before its first shared-memory store; any other row, and a row's last partial
    //    unit, move byte by byte.
    if (tid < kPackRows)
        *reinterpret_cast<uint4*>(&tile[tid][kPadCol]) = make_uint4(0x03030303u, 0x03030303u,
                                                                    0x03030303u, 0x03030303u);
    constexpr int kUnitsPerRow = kChunk / 16;
    constexpr int kLoads = kPackRows * kUnitsPerRow / kPackThreads;   // 8 per thread
    {
        uint4 v[kLoads];
        bool ok[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            const int t = tid + kPackThreads * q;
            const int r = t / kUnitsPerRow, u = t % kUnitsPerRow;
            const int m = m0 + r;
            const uint8_t* p0 = geno + (size_t)(m < M ? m : 0) * N + s0;
            ok[q] = m < M && (reinterpret_cast<uintptr_t>(p0) & 15u) == 0 && 16 * u + 16 <= ns;
            v[q] = ok[q] ? __ldg(reinterpret_cast<const uint4*>(p0) + u) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
            const int t = tid + kPackThreads * q;
            if (ok[q]) {
                bad |= bad_bytes(v[q].x) | bad_bytes(v[q].y) | bad_bytes(v[q].z) | bad_bytes(v[q].w);
                *reinterpret_cast<uint4*>(&tile[t / kUnitsPerRow][16 * (t % kUnitsPerRow)]) = v[q];
            }
        }
    }
    for (int r = wid; r < kPackRows; r += kPackThreads / 32) {
        const int m = m0 + r;
        if (m >= M) continue;   // never stored; its lookups stay inside the tile
        const uint8_t* p0 = geno + (size_t)m * N + s0;
        const int from = (reinterpret_cast<uintptr_t>(p0) & 15u) == 0 ? (ns & ~15) : 0;
        for (int o = from + lane; o < ns; o += 32) {
            const uint32_t g = p0[o];
            bad |= bad_bytes(g);
            tile[r][o] = (uint8_t)g;
        }
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
    const int n0 = ns - total1, n1c = total1;
    const int gl0 = a0 >> 7, gl1 = a1 >> 7;
    const int G0 = n0 ? ((a0 + n0 - 1) >> 7) - gl0 + 1 : 0;
    const int G1 = n1c ? ((a1 + n1c - 1) >> 7) - gl1 + 1 : 0;
    // work items: (group, 32-sample word q), spread evenly over the warps
    const int m = m0 + lane;
    const long long coff0 = pl.coff[0], coff1 = pl.coff[1];
    for (int it = wid; it < 4 * (G0 + G1); it += kPackThreads / 32) {
        const int gi = it >> 2, q = it & 3;
        const int c = gi < G0 ? 0 : 1;
        const int g = c ? gl1 + (gi - G0) : gl0 + gi;
        const int a = c ? a1 : a0, n = c ? n1c : n0;
        const int Nc = c ? N1 : N0;
        const int lo = 128 * g + 32 * q;               // class positions of this word
        if (lo >= Nc || lo + 32 <= a || lo >= a + n) continue;  // pad, or no sample of this chunk
        const bool owned = lo >= a && min(lo + 32, Nc) <= a + n;
        const int loc = lo + lane - a;
        // this lane's sample column (a value-3 column for positions outside this chunk's class)
        const int col = (loc >= 0 && loc < n) ? idx[c][loc] : kPadCol;
        uint32_t w0 = 0u, w1 = 0u;
#pragma unroll 8
        for (int r = 0; r < kPackRows; ++r) {
            const int gv = tile[r][col];
            const uint32_t b0 = __ballot_sync(0xffffffffu, gv == 0);
            const uint32_t b1 = __ballot_sync(0xffffffffu, gv == 1);
            w0 = lane == r ? b0 : w0;
            w1 = lane == r ? b1 : w1;
        }
        if (m < M) {
            const long long coff = c ? coff1 : coff0;
            const int w4 = c ? pl.W4[1] : pl.W4[0];
            uint32_t* e0 = reinterpret_cast<uint32_t*>(planes + coff + (size_t)g * M + m) + q;
            uint32_t* e1 = reinterpret_cast<uint32_t*>(planes + coff + (size_t)(w4 + g) * M + m) + q;
            if (owned) {
                *e0 = w0;
                *e1 = w1;
            } else {
                if (w0) atomicOr(e0, w0);
                if (w1) atomicOr(e1, w1);
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
    static bool carveout = false;  // the whole unified L1 as shared memory: six CTAs per SM
    if (!carveout) {
        e = cudaFuncSetAttribute(pack_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        carveout = true;
    }
    const dim3 grid((N + kChunk - 1) / kChunk, (M + kPackRows - 1) / kPackRows);
    pack_kernel<<<grid, kPackThreads, 0, st>>>(geno, pheno, M, N, counts, N0, N1, pl, planes, ctrl);
    return cudaGetLastError();
}

}  // namespace epi3
