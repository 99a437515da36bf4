// Pairwise (second-order) scan: Eq. 1 applied to two SNPs.  Every pair i < j gets the
// 3^2-cell x {control, case} table and its FP64 K2; the k lowest are returned in the total
// order (K2 ascending, then i, j).
//
// The counts are exact integers straight from the pair tables and marginals built for the
// 8-cell triplet forms: for class c, cells (a, b) with a, b in {0, 1} are the pair table,
//   (a, 2) = n_i(a) - n_ab0 - n_ab1 over b,  (2, b) = n_j(b) - sum over a,
//   (2, 2) = N_c - the other eight.
// The score is summed in cell order 0..8 (cell = 3 gX + gY), term (lf[r+1] - lf[r0]) - lf[r1],
// from the same FP64 log-factorial table as the triplet rescoring, so it equals the oracle's
// bit for bit.  A pair costs 9 x 2 cells: scoring every pair in FP64 is cheap, so no FP32
// band is needed.  Selection: each block scores 2048 consecutive pairs and keeps its k best
// (bitonic sort in shared memory); further passes merge 2048 survivors per block until one
// block remains.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

constexpr int kPairBlock = 2048;      // items sorted per block
constexpr int kPairThreads = 512;     // 4 items per thread

struct Item {
    double s;
    long long key;                    // i * M + j: the tie order (i, j)
};

__device__ __forceinline__ bool item_before(const Item& a, const Item& b) {
    return a.s < b.s || (a.s == b.s && a.key < b.key);
}

// Ascending bitonic sort of kPairBlock items in shared memory (all threads of the block).
__device__ void sort_items(Item* it) {
    for (int size = 2; size <= kPairBlock; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kPairBlock / 2; t += kPairThreads) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const Item x = it[lo], y = it[hi];
                if (item_before(y, x) == up) {
                    it[lo] = y;
                    it[hi] = x;
                }
            }
            __syncthreads();
        }
}

__device__ __forceinline__ Item pad_item() {
    return Item{__longlong_as_double(0x7ff0000000000000LL), 0x7fffffffffffffffLL};  // +inf, last
}

// Pass 1: score pairs [b * 2048, (b + 1) * 2048), keep the block's k best in out[b * k ..].
__global__ void __launch_bounds__(kPairThreads)
pair_score_kernel(PairTables pt, const double* __restrict__ lf64, int M, long long n_pairs,
                  int k, Item* __restrict__ out) {
    __shared__ Item it[kPairBlock];
    const long long p0 = (long long)blockIdx.x * kPairBlock;
    for (int t = threadIdx.x; t < kPairBlock; t += kPairThreads) {
        const long long p = p0 + t;
        if (p >= n_pairs) {
            it[t] = pad_item();
            continue;
        }
        int i, j;
        decode_pair(p, &i, &j);
        double s = 0.0;
        int r[2][9];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int4 q = __ldg(pt.pt + c * pt.n_pairs + p);        // {n00, n01, n10, n11}
            const int2 mi = __ldg(pt.marg + (size_t)c * M + i), mj = __ldg(pt.marg + (size_t)c * M + j);
            r[c][0] = q.x;
            r[c][1] = q.y;
            r[c][2] = mi.x - q.x - q.y;     // (0, 2)
            r[c][3] = q.z;
            r[c][4] = q.w;
            r[c][5] = mi.y - q.z - q.w;     // (1, 2)
            r[c][6] = mj.x - q.x - q.z;     // (2, 0)
            r[c][7] = mj.y - q.y - q.w;     // (2, 1)
            r[c][8] = pt.n_c[c] - (r[c][0] + r[c][1] + r[c][2] + r[c][3] + r[c][4] + r[c][5] +
                                   r[c][6] + r[c][7]);                 // (2, 2)
        }
        // exact counts cannot be negative; a corrupt table is ranked last, never looked up
        int neg = 0;
#pragma unroll
        for (int cell = 0; cell < 9; ++cell) neg |= r[0][cell] | r[1][cell];
        if (neg < 0) {
            it[t] = pad_item();
            continue;
        }
#pragma unroll
        for (int cell = 0; cell < 9; ++cell) {
            const int r0 = r[0][cell], r1 = r[1][cell];
            const double term = __dsub_rn(__dsub_rn(lf64[r0 + r1 + 1], lf64[r0]), lf64[r1]);
            s = __dadd_rn(s, term);
        }
        it[t] = Item{s, (long long)i * M + j};
    }
    __syncthreads();
    sort_items(it);
    for (int t = threadIdx.x; t < k; t += kPairThreads) out[(long long)blockIdx.x * k + t] = it[t];
}

// Merge pass: the k best of each 2048 consecutive survivors.
__global__ void __launch_bounds__(kPairThreads)
pair_merge_kernel(const Item* __restrict__ in, long long n, int k, Item* __restrict__ out) {
    __shared__ Item it[kPairBlock];
    const long long b0 = (long long)blockIdx.x * kPairBlock;
    for (int t = threadIdx.x; t < kPairBlock; t += kPairThreads)
        it[t] = b0 + t < n ? in[b0 + t] : pad_item();
    __syncthreads();
    sort_items(it);
    for (int t = threadIdx.x; t < k; t += kPairThreads) out[(long long)blockIdx.x * k + t] = it[t];
}

__global__ void pair_emit_kernel(const Item* __restrict__ best, int k, int M,
                                 int32_t* __restrict__ out_pairs, double* __restrict__ out_s) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const Item e = best[t];
        out_pairs[2 * t] = (int32_t)(e.key / M);
        out_pairs[2 * t + 1] = (int32_t)(e.key % M);
        out_s[t] = e.s;
    }
}

}  // namespace

size_t pair_scan_scratch(long long n_pairs, int k) {
    const long long blocks = (n_pairs + kPairBlock - 1) / kPairBlock;
    return (size_t)2 * (size_t)blocks * (size_t)k * sizeof(Item);
}

cudaError_t launch_pair_scan(const PairTables& pt, const double* lf64, int M, int k,
                             void* scratch, int32_t* out_pairs, double* out_s, cudaStream_t st) {
    const long long n_pairs = pt.n_pairs;
    long long blocks = (n_pairs + kPairBlock - 1) / kPairBlock;
    Item* a = static_cast<Item*>(scratch);
    Item* b = a + blocks * k;
    pair_score_kernel<<<(unsigned)blocks, kPairThreads, 0, st>>>(pt, lf64, M, n_pairs, k, a);
    cudaError_t e = cudaGetLastError();
    long long n = blocks * k;
    while (e == cudaSuccess && blocks > 1) {
        blocks = (n + kPairBlock - 1) / kPairBlock;
        pair_merge_kernel<<<(unsigned)blocks, kPairThreads, 0, st>>>(a, n, k, b);
        e = cudaGetLastError();
        n = blocks * k;
        Item* t = a;
        a = b;
        b = t;
    }
    if (e != cudaSuccess) return e;
    pair_emit_kernel<<<1, 512, 0, st>>>(a, k, M, out_pairs, out_s);
    return cudaGetLastError();
}

}  // namespace epi3
