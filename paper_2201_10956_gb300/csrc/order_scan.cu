// Scans of other interaction orders: Eq. 1 applied to two, four, five and six SNPs.
//
// Pairs: every pair i < j gets the 3^2-cell x {control, case} table and its FP64 K2; the k
// lowest are returned in the total order (K2 ascending, then i, j).  The counts are exact
// integers straight from the pair tables and marginals built for the 8-cell triplet forms:
// for class c, cells (a, b) with a, b in {0, 1} are the pair table,
//   (a, 2) = n_i(a) - n_ab0 - n_ab1 over b,  (2, b) = n_j(b) - sum over a,
//   (2, 2) = N_c - the other eight.
// The score is summed in cell order 0..8 (cell = 3 gX + gY), term (lf[r+1] - lf[r0]) - lf[r1],
// from the same FP64 log-factorial table as the triplet rescoring, so it equals the oracle's
// bit for bit.  A pair costs 9 x 2 cells: scoring every pair in FP64 is cheap, so no FP32
// band is needed.
//
// Four SNPs: every set i < j < k < l gets its 3^4 = 81-cell table by AND + POPC over the bit
// planes (plane 2 by NOR, pad bits land in cell 80 and are subtracted), built as a product
// tree (3 + 9 + 27 + 81 ANDs per word), both classes' counts packed in one register per cell;
// the FP64 K2 is summed in cell order 0..80 (cell = 27 g_i + 9 g_j + 3 g_k + g_l) like the
// pairs.  The sets are enumerated in colexicographic order from a linear index.
//
// Selection (both): each block scores 2048 consecutive items and keeps its k best (bitonic
// sort in shared memory); further passes merge 2048 survivors per block until one block
// remains.  Ties are ordered by a key that sorts like the SNP indices.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

constexpr int kPairBlock = 2048;      // items sorted per block
constexpr int kPairThreads = 512;     // 4 items per thread
constexpr int kQuadThreads = 256;     // 8 sets per thread (81 packed counters each: registers)

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
            for (int t = threadIdx.x; t < kPairBlock / 2; t += blockDim.x) {
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

// ---------------------------------------------------------------- four SNPs
__host__ __device__ inline long long choose_ll(long long n, int r) {
    if (n < r) return 0;
    long long v = 1;
    for (int t = 0; t < r; ++t) v = v * (n - t) / (t + 1);
    return v;
}

// Largest x in [lo, hi) with choose(x, r) <= q (choose is increasing in x for x >= r - 1).
__device__ inline int colex_digit(long long q, int r, int lo, int hi) {
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (choose_ll(mid, r) <= q) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The q-th 4-set in colexicographic order: q = C(l,4) + C(k,3) + C(j,2) + i, i < j < k < l.
__device__ inline void decode_quad(long long q, int M, int* x) {
    const int l = colex_digit(q, 4, 3, M);
    q -= choose_ll(l, 4);
    const int k = colex_digit(q, 3, 2, l);
    q -= choose_ll(k, 3);
    const int j = colex_digit(q, 2, 1, k);
    q -= choose_ll(j, 2);
    x[0] = (int)q;
    x[1] = j;
    x[2] = k;
    x[3] = l;
}

__device__ __forceinline__ long long quad_key(const int* x) {
    return ((long long)x[0] << 48) | ((long long)x[1] << 32) | ((long long)x[2] << 16) | x[3];
}

// Pass 1 of the four-SNP scan: score sets [b * 2048, (b + 1) * 2048), keep the k best.
__global__ void __launch_bounds__(kQuadThreads)
quad_score_kernel(Planes pl, const double* __restrict__ lf64, int n0, int n1, long long n_sets,
                  int k, Item* __restrict__ out) {
    __shared__ Item it[kPairBlock];
    const long long q0 = (long long)blockIdx.x * kPairBlock;
    const int M = pl.M;
    for (int t = threadIdx.x; t < kPairBlock; t += kQuadThreads) {
        const long long q = q0 + t;
        if (q >= n_sets) {
            it[t] = pad_item();
            continue;
        }
        int x[4];
        decode_quad(q, M, x);
        // cnt[cell] = count of class 0 + (count of class 1 << 16)
        uint32_t cnt[81];
#pragma unroll
        for (int cell = 0; cell < 81; ++cell) cnt[cell] = 0u;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const long long coff = c ? pl.coff[1] : pl.coff[0];
            const int W4 = c ? pl.W4[1] : pl.W4[0];
            const int sh = 16 * c;
#pragma unroll 1
            for (int w4 = 0; w4 < W4; ++w4) {
                uint4 g0[4], g1[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    g0[v] = __ldg(pl.planes + coff + (size_t)w4 * M + x[v]);
                    g1[v] = __ldg(pl.planes + coff + (size_t)(W4 + w4) * M + x[v]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t P[4][3];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const uint32_t a0 = e == 0 ? g0[v].x : e == 1 ? g0[v].y : e == 2 ? g0[v].z : g0[v].w;
                        const uint32_t a1 = e == 0 ? g1[v].x : e == 1 ? g1[v].y : e == 2 ? g1[v].z : g1[v].w;
                        P[v][0] = a0;
                        P[v][1] = a1;
                        P[v][2] = ~(a0 | a1);        // genotype 2, Sec. IV-A (pad bits read 2)
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            const uint32_t ab = P[0][a] & P[1][b];
#pragma unroll
                            for (int cc = 0; cc < 3; ++cc) {
                                const uint32_t abc = ab & P[2][cc];
#pragma unroll
                                for (int d = 0; d < 3; ++d)
                                    cnt[27 * a + 9 * b + 3 * cc + d] +=
                                        (uint32_t)__popc(abc & P[3][d]) << sh;
                            }
                        }
                }
            }
        }
        // pad samples read genotype 2 in all four SNPs: cell (2, 2, 2, 2) only
        cnt[80] -= (uint32_t)pl.pad[0] + ((uint32_t)pl.pad[1] << 16);
        double s = 0.0;
#pragma unroll
        for (int cell = 0; cell < 81; ++cell) {
            const int r0 = (int)(cnt[cell] & 0xFFFFu), r1 = (int)(cnt[cell] >> 16);
            const double term = __dsub_rn(__dsub_rn(lf64[r0 + r1 + 1], lf64[r0]), lf64[r1]);
            s = __dadd_rn(s, term);
        }
        (void)n0;
        (void)n1;
        it[t] = Item{s, quad_key(x)};
    }
    __syncthreads();
    sort_items(it);
    for (int t = threadIdx.x; t < k; t += kQuadThreads) out[(long long)blockIdx.x * k + t] = it[t];
}

__global__ void quad_emit_kernel(const Item* __restrict__ best, int k, int32_t* __restrict__ out_snps,
                                 double* __restrict__ out_s) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const Item e = best[t];
        out_snps[4 * t] = (int32_t)((e.key >> 48) & 0xFFFF);
        out_snps[4 * t + 1] = (int32_t)((e.key >> 32) & 0xFFFF);
        out_snps[4 * t + 2] = (int32_t)((e.key >> 16) & 0xFFFF);
        out_snps[4 * t + 3] = (int32_t)(e.key & 0xFFFF);
        out_s[t] = e.s;
    }
}

// ---------------------------------------------------------------- five and six SNPs
// The same table and score for order K = 5, 6 (3^K = 243, 729 cells), one warp per set: lane l
// owns cells l, l + 32, ..., each cell's genotype digits kept as 2-bit codes (x_0 most
// significant, as in the cell index); per 32-sample word every lane ANDs the K plane words its
// cells select and adds the POPC (both classes packed in one counter, class 1 in the high
// half).  The FP64 K2 is then summed in cell order 0 .. 3^K - 1 by every lane from the lanes'
// terms (warp shuffles in cell order), as the oracle adds them.  Sets are enumerated in
// lexicographic order, so the rank q itself is the tie key.
constexpr int kOrdThreads = 256;      // 8 warps per block, 256 sets each

template <int K>
struct Pow3 {
    static constexpr int v = 3 * Pow3<K - 1>::v;
};
template <>
struct Pow3<0> {
    static constexpr int v = 1;
};

// The q-th K-set x_0 < ... < x_{K-1} of M SNPs in lexicographic order.
template <int K>
__device__ inline void decode_lex(long long q, int M, int* x) {
    int v = 0;
#pragma unroll
    for (int t = 0; t < K; ++t)
        for (;; ++v) {
            const long long c = choose_ll(M - 1 - v, K - 1 - t);   // sets with x_t = v
            if (q < c) {
                x[t] = v++;
                break;
            }
            q -= c;
        }
}

template <int K>
__global__ void __launch_bounds__(kOrdThreads)
order_score_kernel(Planes pl, const double* __restrict__ lf64, long long n_sets, int k,
                   Item* __restrict__ out) {
    constexpr int kCellsK = Pow3<K>::v, kPer = (kCellsK + 31) / 32;
    __shared__ Item it[kPairBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int M = pl.M;
    uint32_t code[kPer];   // 2 bits per SNP: the genotype of x_t at bits 2 t
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
        int e = lane + 32 * m < kCellsK ? lane + 32 * m : 0;
        uint32_t cd = 0u;
#pragma unroll
        for (int t = K - 1; t >= 0; --t) {
            cd |= (uint32_t)(e % 3) << (2 * t);
            e /= 3;
        }
        code[m] = cd;
    }
    const long long q0 = (long long)blockIdx.x * kPairBlock;
    for (int t = warp; t < kPairBlock; t += kOrdThreads / 32) {
        const long long q = q0 + t;
        if (q >= n_sets) {   // uniform over the warp
            if (lane == 0) it[t] = pad_item();
            continue;
        }
        int x[K];
        decode_lex<K>(q, M, x);
        uint32_t cnt[kPer];
#pragma unroll
        for (int m = 0; m < kPer; ++m) cnt[m] = 0u;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const long long coff = c ? pl.coff[1] : pl.coff[0];
            const int W4 = c ? pl.W4[1] : pl.W4[0];
            const int sh = 16 * c;
#pragma unroll 1
            for (int w4 = 0; w4 < W4; ++w4) {
                uint4 g0[K], g1[K];
#pragma unroll
                for (int v = 0; v < K; ++v) {
                    g0[v] = __ldg(pl.planes + coff + (size_t)w4 * M + x[v]);
                    g1[v] = __ldg(pl.planes + coff + (size_t)(W4 + w4) * M + x[v]);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t P[K][3];
#pragma unroll
                    for (int v = 0; v < K; ++v) {
                        const uint32_t a0 = e == 0 ? g0[v].x : e == 1 ? g0[v].y : e == 2 ? g0[v].z : g0[v].w;
                        const uint32_t a1 = e == 0 ? g1[v].x : e == 1 ? g1[v].y : e == 2 ? g1[v].z : g1[v].w;
                        P[v][0] = a0;
                        P[v][1] = a1;
                        P[v][2] = ~(a0 | a1);        // genotype 2, Sec. IV-A (pad bits read 2)
                    }
#pragma unroll
                    for (int m = 0; m < kPer; ++m) {
                        uint32_t acc = 0xFFFFFFFFu;
#pragma unroll
                        for (int v = 0; v < K; ++v) {
                            const uint32_t g = (code[m] >> (2 * v)) & 3u;
                            acc &= g == 0u ? P[v][0] : (g == 1u ? P[v][1] : P[v][2]);
                        }
                        cnt[m] += (uint32_t)__popc(acc) << sh;
                    }
                }
            }
        }
        // pad samples read genotype 2 in every SNP: the last cell only
        if (lane == (kCellsK - 1) % 32)
            cnt[(kCellsK - 1) / 32] -= (uint32_t)pl.pad[0] + ((uint32_t)pl.pad[1] << 16);
        double term[kPer];
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
            const int r0 = (int)(cnt[m] & 0xFFFFu), r1 = (int)(cnt[m] >> 16);
            term[m] = lane + 32 * m < kCellsK
                          ? __dsub_rn(__dsub_rn(lf64[r0 + r1 + 1], lf64[r0]), lf64[r1]) : 0.0;
        }
        double sc = 0.0;
#pragma unroll
        for (int m = 0; m < kPer; ++m)
#pragma unroll
            for (int l = 0; l < 32; ++l)
                if (32 * m + l < kCellsK) sc = __dadd_rn(sc, __shfl_sync(0xffffffffu, term[m], l));
        if (lane == 0) it[t] = Item{sc, q};
    }
    __syncthreads();
    sort_items(it);
    for (int t = threadIdx.x; t < k; t += kOrdThreads) out[(long long)blockIdx.x * k + t] = it[t];
}

template <int K>
__global__ void order_emit_kernel(const Item* __restrict__ best, int k, int M,
                                  int32_t* __restrict__ out_snps, double* __restrict__ out_s) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const Item e = best[t];
        int x[K];
        decode_lex<K>(e.key, M, x);
#pragma unroll
        for (int v = 0; v < K; ++v) out_snps[K * t + v] = (int32_t)x[v];
        out_s[t] = e.s;
    }
}

template <int K>
cudaError_t order_scan_k(const Planes& pl, const double* lf64, int k, void* scratch,
                         int32_t* out_snps, double* out_s, cudaStream_t st) {
    const long long n_sets = choose_ll(pl.M, K);
    long long blocks = (n_sets + kPairBlock - 1) / kPairBlock;
    Item* a = static_cast<Item*>(scratch);
    Item* b = a + blocks * k;
    order_score_kernel<K><<<(unsigned)blocks, kOrdThreads, 0, st>>>(pl, lf64, n_sets, k, a);
    cudaError_t e = cudaGetLastError();
    long long n = blocks * k;
    while (e == cudaSuccess && blocks > 1) {
        blocks = (n + kPairBlock - 1) / kPairBlock;
        pair_merge_kernel<<<(unsigned)blocks, kPairThreads, 0, st>>>(a, n, k, b);
        e = cudaGetLastError();
        n = blocks * k;
        Item* tmp = a;
        a = b;
        b = tmp;
    }
    if (e != cudaSuccess) return e;
    order_emit_kernel<K><<<1, 512, 0, st>>>(a, k, pl.M, out_snps, out_s);
    return cudaGetLastError();
}

}  // namespace

long long order_count(int M, int order) { return choose_ll(M, order); }

size_t order_scan_scratch(int M, int order, int k) {
    const long long blocks = (choose_ll(M, order) + kPairBlock - 1) / kPairBlock;
    return (size_t)2 * (size_t)blocks * (size_t)k * sizeof(Item);
}

cudaError_t launch_order_scan(const Planes& pl, const double* lf64, int order, int k, void* scratch,
                              int32_t* out_snps, double* out_s, cudaStream_t st) {
    if (order == 5) return order_scan_k<5>(pl, lf64, k, scratch, out_snps, out_s, st);
    if (order == 6) return order_scan_k<6>(pl, lf64, k, scratch, out_snps, out_s, st);
    return cudaErrorInvalidValue;
}

long long quad_count(int M) { return choose_ll(M, 4); }

size_t quad_scan_scratch(int M, int k) {
    const long long blocks = (choose_ll(M, 4) + kPairBlock - 1) / kPairBlock;
    return (size_t)2 * (size_t)blocks * (size_t)k * sizeof(Item);
}

cudaError_t launch_quad_scan(const Planes& pl, const double* lf64, int n0, int n1, int k,
                             void* scratch, int32_t* out_snps, double* out_s, cudaStream_t st) {
    const long long n_sets = choose_ll(pl.M, 4);
    long long blocks = (n_sets + kPairBlock - 1) / kPairBlock;
    Item* a = static_cast<Item*>(scratch);
    Item* b = a + blocks * k;
    quad_score_kernel<<<(unsigned)blocks, kQuadThreads, 0, st>>>(pl, lf64, n0, n1, n_sets, k, a);
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
    quad_emit_kernel<<<1, 512, 0, st>>>(a, k, out_snps, out_s);
    return cudaGetLastError();
}

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
