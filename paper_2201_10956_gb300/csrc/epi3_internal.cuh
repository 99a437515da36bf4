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
constexpr int kStTimeout = 64;
constexpr int kStBadCount = 128;  // a tensor-core table failed its range check

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
    // first bounded wait that ran out (0 = none): role + 1, then the tile, set and step it
    // was on (diagnostics of EPI3_ERR_TIMEOUT)
    unsigned int wait_role, wait_tile, wait_set, wait_step;
    unsigned int pad_[3];
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
    // |K2 bound - s32| <= prune_delta for every table of this data set (0: no pruning)
    float prune_delta;
};

// Pair tables for the 8-cell forms: for SNPs m1 < m2 (pair index p = m2(m2-1)/2 + m1)
// and class c, pt[c * n_pairs + p] = {n00, n01, n10, n11}, nab = samples with genotype a at
// m1 and b at m2; marg[c * M + m] = {n0, n1}; n_c = class sizes.
struct PairTables {
    const int4* pt;
    const int2* marg;
    long long n_pairs;
    int n_c[2];
    // the tensor scan's copies in FP32 (exact), offset for its count + 1 arithmetic: every
    // pair-table entry + 3, every marginal + 9 (null until that scan needs them)
    const float4* ptf;
    const float2* margf;
};

struct ScanArgs {
    Planes pl;
    K2Tables k2;
    PairTables pt;
    Ctrl* ctrl;
    Cand* cand;
    long long cand_cap;
    long long pair_begin, pair_end;
    int top_k;
    float* dbg;                   // optional: FP32 score of every triplet at (i*M + j)*M + k
    unsigned long long* tsum;     // optional: table checksum slots (table_sum), no pruning
};

// launchers (return cudaError_t of the launch)
// counts[0] = controls, counts[1] = cases, counts[2 + q] = cases before sample 1024 q
// (class_counts_len(N) ints); the pack kernel reads them to place each chunk's samples.
size_t class_counts_len(int N);
cudaError_t launch_class_index(const uint8_t* pheno, int N, int* counts, Ctrl* ctrl,
                               cudaStream_t st);
// zeroes the planes, then packs (both on st)
cudaError_t launch_pack(const uint8_t* geno, const uint8_t* pheno, int M, int N, const int* counts,
                        int N0, int N1, const Planes& pl, uint4* planes, Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_scan_popc(const ScanArgs& a, int grid, int block, size_t smem, cudaStream_t st);
size_t scan_popc_smem(const Planes& pl);
cudaError_t scan_popc_occupancy(int block, size_t smem, int* ctas_per_sm);
cudaError_t launch_select(Ctrl* ctrl, const Cand* cand, long long cand_cap, int top_k,
                          float rel, float abs_, cudaStream_t st);
cudaError_t launch_rescore(const Planes& pl, const K2Tables& k2, Ctrl* ctrl, const Cand* cand,
                           long long cand_cap, Final* fin, int grid, cudaStream_t st);
cudaError_t launch_final(Ctrl* ctrl, const Final* fin, int top_k, double* out_scores,
                         int* out_trip, cudaStream_t st);
cudaError_t launch_tables(const Planes& pl, const PairTables* pt, const K2Tables* k2, long long n,
                          const int* trip, int* out_counts, float* out_s32, double* out_s64,
                          Ctrl* ctrl, cudaStream_t st);
cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st);
// Pairwise scan (Eq. 1 for two SNPs): the k best pairs by (FP64 K2, i, j) from the pair tables.
size_t pair_scan_scratch(long long n_pairs, int k);
cudaError_t launch_pair_scan(const PairTables& pt, const double* lf64, int M, int k,
                             void* scratch, int32_t* out_pairs, double* out_s, cudaStream_t st);
// Four-SNP scan (Eq. 1 for four SNPs, 81 cells): the k best sets by (FP64 K2, i, j, k, l) from
// the bit planes; needs both class sizes below 65536 and M below 65536.
// orders 5 and 6: every set by AND + POPC (one warp per set), FP64 K2 in cell order
long long order_count(int M, int order);
size_t order_scan_scratch(int M, int order, int k);
cudaError_t launch_order_scan(const Planes& pl, const double* lf64, int order, int k, void* scratch,
                              int32_t* out_snps, double* out_s, cudaStream_t st);
long long quad_count(int M);
size_t quad_scan_scratch(int M, int k);
cudaError_t launch_quad_scan(const Planes& pl, const double* lf64, int n0, int n1, int k,
                             void* scratch, int32_t* out_snps, double* out_s, cudaStream_t st);
// max over n in [0, n_lf) of (n + 1/2) |lg2_hw(n + 1) - log2(n + 1)| (FP64) into *out (device).
cudaError_t launch_approx_error(const double* lf64, int n_lf, double* out, cudaStream_t st);
cudaError_t launch_pair_tables(const Planes& pl, int4* pt, int2* marg, long long n_pairs,
                               cudaStream_t st);
// ptf = pt + 3 and margf = marg + 9 as FP32 (2 n_pairs and 2 M entries)
cudaError_t launch_pair_floats(const int4* pt, const int2* marg, long long n_pairs, int M,
                               float4* ptf, float2* margf, cudaStream_t st);
cudaError_t launch_scan_popc8(const ScanArgs& a, int grid, int block, size_t smem, cudaStream_t st);
size_t scan_popc8_smem(const Planes& pl);
size_t scan_mma_smem(int kind);
// Element kinds of the tensor-core scan's 0/1 operands: FP16, FP8 E4M3, block-scaled FP4 E2M1
// (two per byte).  A 128-byte operand row holds 64, 128 or 256 samples.
enum { kKindF16 = 0, kKindE4M3 = 1, kKindE2M1 = 2 };
int mma_samples_per_step(int kind);
// Tensor-scan tiles of a whole scan built on the device: blocks[b] = {kb, jb, count, offset},
// tiles (i, jb, kb, cohort) for i < count written from offset on.
cudaError_t launch_tile_list(const int4* blocks, int n_blocks, int cohort, int4* tiles,
                             cudaStream_t st);
cudaError_t launch_onehot(const Planes& pl, uint8_t* oh, long long off1, int KS0, int KS1,
                          int kb_count, int kind, cudaStream_t st);
// bytes of the one-hot chunks and their two rearranged views (one allocation: oh | yoh | xoh)
size_t onehot_bytes(int M, int KS0, int KS1);
cudaError_t launch_onehot_views(const uint8_t* oh, long long off1, int KS0, int KS1, int kb_count,
                                int M, uint8_t* yoh, uint8_t* xoh, cudaStream_t st);
// One data set ("cohort") as the tensor-core scan sees it.  The kernel reads these from
// device memory, one per tile (tile.w = cohort index), so one launch can scan many.
struct CohortDev {
    Planes pl;
    K2Tables k2;
    PairTables pt;
    const uint8_t* oh;        // pre-tiled one-hot chunks [class][64-SNP block][K-step], 16 KB
    long long oh_off1;        // chunk index of class 1 (class 0 starts at 0)
    const uint8_t* yoh;       // second-SNP rows [class][32-SNP block][K-step], 8 KB each
    long long yoh_off1;       // 8 KB unit of class 1
    const uint8_t* xoh;       // first-SNP rows [class][SNP][K-step], 256 B each
    long long xoh_off1;       // 256 B unit of class 1
    int KS[2];                // K-steps per class
    long long pair_begin, pair_end;
    Ctrl* ctrl;
    Cand* cand;
    long long cand_cap;
    int top_k;
    float* dbg;
    unsigned long long* tsum;     // optional: table checksum slots (table_sum), no pruning
    int inject_timeout;       // test hook: the MMA issuer first waits on a barrier nobody signals
};

// ---------------------------------------------------------------- sample-compacted tensor scan
constexpr int kCmpSets = 4;      // (class, one of the two counted genotypes of the first SNP)
// Per first SNP of a compaction range: the chunk index of (block b_lo, step 0) of each set and
// the sets' K-steps; chunk (b, ks) of set q is base[q] + (b - b_lo) * ks[q] + ks.  The first
// SNP's most frequent genotype (over both classes) is derived, not counted: set 2 c + s holds
// the class-c samples whose first-SNP genotype is cmp_geno(drop, s).  Both classes derive the
// same genotype, so that every cell of one class meets the same cell of the other.
struct CmpFirst {
    long long base[kCmpSets];
    int ks[kCmpSets];
    int drop;
    int b_lo;                    // first 64-SNP block compacted: the first j block of the tiles
    int tiles;                   // tiles of this first SNP
    int jb_end;                  // one past its last j block (the pair range's last j)
    long long tile0;             // index of its first tile in the range
};

struct CmpArgs {
    CohortDev cd;                // tables, candidate stage, pair range, test hooks
    const CmpFirst* firsts;      // per first SNP of the range
    int i0, n_first;
    long long n_tiles;           // tiles of the range
    const uint8_t* cmp;          // compacted chunks of the range
    unsigned long long* prof;    // optional (instrumented kernel): wait cycles per role
};
// The genotype counted in slot s (0, 1) when genotype d is derived: the other two, ascending.
__host__ __device__ __forceinline__ int cmp_geno(int d, int s) {
    return s == 0 ? (d == 0 ? 1 : 0) : (d == 2 ? 1 : 2);
}
// The genotype derived: the most frequent one (ties: 2, then 0), so that the two counted sets
// are the smallest; n0, n1, n2 = counts of genotypes 0, 1, 2 over both classes.
inline int cmp_drop(int n0, int n1, int n2) {
    if (n2 >= n0 && n2 >= n1) return 2;
    return n0 >= n1 ? 0 : 1;
}
// A first SNP whose derived genotype d is not 2 counts the other two: slot s = 0, 1 holds
// genotype cmp_geno(d, s) and the derived genotype takes label 2 (in both classes alike), so the
// tensor scan's inclusion-exclusion and bound run unchanged on relabelled inputs (every value an
// exact integer; the bound is a sum over cells, each cell pairing its two classes).
// Pair table (X = first SNP, W) of a class, n(a, w) at 2 a + w, with W's marginal {n0, n1}.
__host__ __device__ __forceinline__ int4 relabel_xy(int4 p, int2 mw, int d) {
    const int n20 = mw.x - p.x - p.z, n21 = mw.y - p.y - p.w;
    return d == 0 ? make_int4(p.z, p.w, n20, n21) : d == 1 ? make_int4(p.x, p.y, n20, n21) : p;
}
// Marginal of the first SNP {n0, n1} in a class of nc samples.
__host__ __device__ __forceinline__ int2 relabel_marg(int2 m, int nc, int d) {
    const int n2 = nc - m.x - m.y;
    return d == 0 ? make_int2(m.y, n2) : d == 1 ? make_int2(m.x, n2) : m;
}
// The same for the FP32 pair-table row (X, Z) (+ 3 each, index 2 a + z) with Z's marginal + 9
// (exact: integers below 2^24).
__host__ __device__ __forceinline__ float4 relabel_xz(float4 x, float2 mz9, int d) {
    if (d == 2) return x;
    const float r0 = (mz9.x - x.x) - x.z, r1 = (mz9.y - x.y) - x.w;
    return d == 0 ? make_float4(x.z, x.w, r0, r1) : make_float4(x.x, x.y, r0, r1);
}
// Cells u[9 a + 3 b + z] of relabelled first-SNP genotypes back in genotype order.
template <class T>
__host__ __device__ __forceinline__ void canon_rows(T* u, int d) {
    if (d == 2) return;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        const T r0 = u[e], r1 = u[9 + e], r2 = u[18 + e];   // slot 0, slot 1, derived
        if (d == 0) {            // genotypes 1, 2, 0
            u[e] = r2;
            u[9 + e] = r0;
            u[18 + e] = r1;
        } else {                 // genotypes 0, 2, 1
            u[9 + e] = r2;
            u[18 + e] = r1;
        }
    }
}
// compacted chunks of one first SNP: 16 KB each
inline long long cmp_chunks_of(const CmpFirst& f, int M) {
    const long long nblk = (M + 63) / 64 - f.b_lo;
    return nblk * ((long long)f.ks[0] + f.ks[1] + f.ks[2] + f.ks[3]);
}
int cmp_tiles_of(int M, int b_lo, int jb_end); // tiles (64 j x 32 k) of one first SNP
size_t scan_cmp_smem();
// compaction of first SNPs i0 .. i0 + n_first - 1 into cmp (chunk indices from firsts)
cudaError_t launch_compact(const Planes& pl, const CmpFirst* firsts, int i0, int n_first,
                           uint8_t* cmp, cudaStream_t st);
// instrumented: table checksums / wait profile; paired: the two-triplets-per-lane epilogue
cudaError_t launch_scan_cmp(const CmpArgs& a, int grid, cudaStream_t st, bool instrumented, bool paired);

// tiles[t] = (i, j-block, k-block, cohort); a CTA takes tiles blockIdx.x, +gridDim.x, ...
// split: the register-split form of the kernel (measured per shape by the handle tuner, per
// batch by timing both forms on its first scan)
// checksum: the cohorts' tsum slots are set (the instrumented instantiation adds every table)
cudaError_t launch_scan_mma(const CohortDev* cohorts, const int4* tiles, long long n_tiles,
                            int kind, int grid, cudaStream_t st, unsigned long long* prof,
                            bool split, bool checksum = false);
int mma_threads(bool split);   // threads per CTA of the tensor-core scan
cudaError_t scan_popc8_occupancy(int block, size_t smem, int* ctas_per_sm);

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

__host__ __device__ inline long long pair_index(int m1, int m2) {  // m1 < m2
    return (long long)m2 * (m2 - 1) / 2 + m1;
}

// The 27 cells of one class from the 8 cells with every genotype in {0, 1}, by exact
// integer inclusion-exclusion over the pair tables and single-SNP marginals (a cell with
// genotype 2 at one SNP is the pair count minus the two cells with 0 and 1 there).
//   n8[4a + 2b + z] = #(gX = a, gY = b, gZ = z);  pxy = (X, Y) pair table {n00,n01,n10,n11},
//   pxz = (X, Z), pyz = (Y, Z);  mx, my, mz = {n0, n1};  nc = class size.
//   r[9 gX + 3 gY + gZ] for gX, gY, gZ in {0, 1, 2}.
__host__ __device__ __forceinline__ void derive27(const int* n8, int4 pxy, int4 pxz, int4 pyz,
                                                  int2 mx, int2 my, int2 mz, int nc, int* r) {
    const int xy[2][2] = {{pxy.x, pxy.y}, {pxy.z, pxy.w}};
    const int xz[2][2] = {{pxz.x, pxz.y}, {pxz.z, pxz.w}};
    const int yz[2][2] = {{pyz.x, pyz.y}, {pyz.z, pyz.w}};
    const int mxa[2] = {mx.x, mx.y}, myb[2] = {my.x, my.y}, mzc[2] = {mz.x, mz.y};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int c0 = n8[4 * a + 2 * b], c1 = n8[4 * a + 2 * b + 1];
            r[9 * a + 3 * b + 0] = c0;
            r[9 * a + 3 * b + 1] = c1;
            r[9 * a + 3 * b + 2] = xy[a][b] - c0 - c1;                     // (a, b, 2)
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int z = 0; z < 2; ++z) r[9 * a + 6 + z] = xz[a][z] - r[9 * a + z] - r[9 * a + 3 + z];  // (a,2,z)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int z = 0; z < 2; ++z) r[18 + 3 * b + z] = yz[b][z] - r[3 * b + z] - r[9 + 3 * b + z];  // (2,b,z)
#pragma unroll
    for (int a = 0; a < 2; ++a)  // (a, 2, 2): pair (X,Y) count at (a, 2) minus (a,2,0), (a,2,1)
        r[9 * a + 8] = (mxa[a] - xy[a][0] - xy[a][1]) - r[9 * a + 6] - r[9 * a + 7];
#pragma unroll
    for (int b = 0; b < 2; ++b)  // (2, b, 2)
        r[18 + 3 * b + 2] = (myb[b] - xy[0][b] - xy[1][b]) - r[18 + 3 * b] - r[18 + 3 * b + 1];
#pragma unroll
    for (int z = 0; z < 2; ++z)  // (2, 2, z)
        r[24 + z] = (mzc[z] - xz[0][z] - xz[1][z]) - r[18 + z] - r[21 + z];
    int s = 0;
#pragma unroll
    for (int q = 0; q < 26; ++q) s += r[q];
    r[26] = nc - s;                                                       // (2, 2, 2)
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

// Table-free approximate K2 (the tensor scan's pruning bound), used only to prove that a table
// lies above the candidate band.
// Stirling: lf(n) = (n + 1/2) ln(n + 1) - (n + 1) + ln(2 pi)/2 + e(n), 0 < e(n) <= 1/(12(n+1)).
// In a cell term lf(r+1) - lf(r0) - lf(r1) (r = r0 + r1) the linear parts cancel, so
//   K2 ~= ln 2 * sum_c [phi(r+1) - phi(r0) - phi(r1)] - 27 ln(2 pi)/2,  phi(n) = (n+1/2) log2(n+1),
// off by the Stirling remainders (at most 1/6 per cell), by the error of this hardware log2
// inside phi (measured for every n of a data set by launch_approx_error) and by the FP32
// rounding of the FMA chains.  Every operation is an explicit intrinsic, so the value does not
// depend on the compiler's contraction choices.
__device__ __forceinline__ float lg2_hw(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// n as FP32, exact for 0 <= n < 2^23 (n + 2^23 has the integer in its mantissa)
__device__ __forceinline__ float exact_float(int n) {
    return __fsub_rn(__int_as_float(n + 0x4B000000), 8388608.0f);
}

// Order-independent checksum of counted tables (debug entry point epi3_scan_checksum): every
// table's hash(i, j, k, r0, r1) is summed (mod 2^64) by the thread that counted it, and each
// thread adds its sum and its table count into one of kTsumSlots slot pairs at the end; the
// host sums the slots.  The hash is the splitmix64 finaliser applied to a multiply-add fold of
// the 54 counts and to the packed triplet key.
constexpr int kTsumSlots = 32;
__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ inline unsigned long long table_hash(int i, int j, int k, const int* r0, const int* r1) {
    unsigned long long f = 0;
    for (int q = 0; q < kCells; ++q)
        f = f * 0x100000001B3ull + (unsigned long long)(unsigned)r0[q] +
            ((unsigned long long)(unsigned)r1[q] << 32);
    return mix64(f ^ mix64(pack_key(i, j, k)));
}
__device__ inline void table_sum_flush(unsigned long long* tsum, unsigned long long h,
                                       unsigned long long n) {
    if (n == 0) return;
    const int slot = (int)((threadIdx.x + blockIdx.x) % kTsumSlots);
    atomicAdd(tsum + slot, h);
    atomicAdd(tsum + kTsumSlots + slot, n);
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
