// Candidate stage of the scan and the per-triplet debug kernels.
//
//   reset    : zero the control block, threshold = +inf.
//   select   : exact k-th smallest FP32 score among the global candidates (radix select
//              on the float bit patterns, which order like the non-negative values), then
//              the rescoring band T = band_threshold(k-th).
//   rescore  : one warp per candidate inside the band: recount its 2 x 27 table (lanes
//              split the sample groups, warp-shuffle sums of the 54 counts), FP64 K2
//              (Eq. 1, cell order 0..26).
//   final    : one CTA sorts the rescored candidates by (K2, i, j, k) and writes the
//              first top_k (Sec. III: the lowest K2 is the solution).
//   tables   : warp per listed triplet, tables and/or FP32 and FP64 K2.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

constexpr int kSelThreads = 1024;
constexpr int kFinThreads = 1024;

__device__ __forceinline__ int popc4(uint4 a, uint4 b, uint4 c) {
    return __popc(a.x & b.x & c.x) + __popc(a.y & b.y & c.y) + __popc(a.z & b.z & c.z) +
           __popc(a.w & b.w & c.w);
}

__device__ __forceinline__ uint4 nor4(uint4 a, uint4 b) {
    return make_uint4(~(a.x | b.x), ~(a.y | b.y), ~(a.z | b.z), ~(a.w | b.w));
}

// Exact table of (x, y, z) by one warp: lanes take 128-sample groups, then butterfly sums.
// On return every lane holds r0[27] (controls) and r1[27] (cases).
__device__ void warp_table(const Planes& pl, int x, int y, int z, int* r0, int* r1) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        int* r = c ? r1 : r0;
#pragma unroll
        for (int q = 0; q < kCells; ++q) r[q] = 0;
        const int W4 = pl.W4[c];
        const uint4* base = pl.planes + pl.coff[c];
        const size_t ps = (size_t)W4 * pl.M;
        for (int w4 = lane; w4 < W4; w4 += 32) {
            const size_t o = (size_t)w4 * pl.M;
            uint4 X[3], Y[3], Z[3];
            X[0] = __ldg(base + o + x); X[1] = __ldg(base + ps + o + x); X[2] = nor4(X[0], X[1]);
            Y[0] = __ldg(base + o + y); Y[1] = __ldg(base + ps + o + y); Y[2] = nor4(Y[0], Y[1]);
            Z[0] = __ldg(base + o + z); Z[1] = __ldg(base + ps + o + z); Z[2] = nor4(Z[0], Z[1]);
#pragma unroll
            for (int gx = 0; gx < 3; ++gx)
#pragma unroll
                for (int gy = 0; gy < 3; ++gy)
#pragma unroll
                    for (int gz = 0; gz < 3; ++gz) r[9 * gx + 3 * gy + gz] += popc4(X[gx], Y[gy], Z[gz]);
        }
#pragma unroll
        for (int q = 0; q < kCells; ++q) {
            int v = r[q];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            r[q] = v;
        }
        r[kCells - 1] -= pl.pad[c];
    }
}

// 8-cell form of warp_table: counts the cells with genotypes in {0,1} and derives the
// other 19 from the pair tables (derive27).
__device__ void warp_table8(const Planes& pl, const PairTables& pt, int x, int y, int z, int* r0,
                            int* r1) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        int n8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) n8[q] = 0;
        const int W4 = pl.W4[c];
        const uint4* base = pl.planes + pl.coff[c];
        const size_t ps = (size_t)W4 * pl.M;
        for (int w4 = lane; w4 < W4; w4 += 32) {
            const size_t o = (size_t)w4 * pl.M;
            const uint4 X[2] = {__ldg(base + o + x), __ldg(base + ps + o + x)};
            const uint4 Y[2] = {__ldg(base + o + y), __ldg(base + ps + o + y)};
            const uint4 Z[2] = {__ldg(base + o + z), __ldg(base + ps + o + z)};
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int g = 0; g < 2; ++g) n8[4 * a + 2 * b + g] += popc4(X[a], Y[b], Z[g]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int v = n8[q];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            n8[q] = v;
        }
        // pair tables are stored for ordered pairs m1 < m2; swap roles when needed
        auto pair = [&](int u, int v) -> int4 {
            if (u < v) return __ldg(pt.pt + c * pt.n_pairs + pair_index(u, v));
            const int4 t = __ldg(pt.pt + c * pt.n_pairs + pair_index(v, u));
            return make_int4(t.x, t.z, t.y, t.w);  // transpose the 2 x 2 table
        };
        derive27(n8, pair(x, y), pair(x, z), pair(y, z), __ldg(pt.marg + (size_t)c * pl.M + x),
                 __ldg(pt.marg + (size_t)c * pl.M + y), __ldg(pt.marg + (size_t)c * pl.M + z),
                 pt.n_c[c], c ? r1 : r0);
    }
}

__global__ void reset_kernel(Ctrl* ctrl) {
    Ctrl z = {};
    z.thr = 0x7f800000u;
    *ctrl = z;
}

__global__ void __launch_bounds__(kSelThreads)
select_kernel(Ctrl* ctrl, const Cand* __restrict__ cand, long long cap, int top_k, float rel,
              float abs_) {
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_rank;
    const int tid = threadIdx.x;
    const long long n = min((long long)ctrl->n_cand, cap);
    if (n < top_k) {
        if (tid == 0) atomicOr(&ctrl->status, kStInternal);
        return;
    }
    if (tid == 0) {
        s_prefix = 0u;
        s_rank = (unsigned)top_k;  // 1-based rank still to find inside the current prefix
    }
    unsigned mask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += kSelThreads) hist[b] = 0u;
        __syncthreads();
        const unsigned prefix = s_prefix;
        for (long long idx = tid; idx < n; idx += kSelThreads) {
            const unsigned u = __float_as_uint(cand[idx].s);
            if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned cum = 0u, rank = s_rank;
            int digit = 255;
            for (int b = 0; b < 256; ++b) {
                if (cum + hist[b] >= rank) {
                    digit = b;
                    break;
                }
                cum += hist[b];
            }
            s_rank = rank - cum;
            s_prefix = prefix | ((unsigned)digit << shift);
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    if (tid == 0) {
        const float kth = __uint_as_float(s_prefix);
        ctrl->kth = kth;
        ctrl->t_final = band_threshold(kth, rel, abs_);
    }
}

__global__ void __launch_bounds__(256)
rescore_kernel(Planes pl, K2Tables k2, Ctrl* ctrl, const Cand* __restrict__ cand, long long cap,
               Final* __restrict__ fin) {
    const long long n = min((long long)ctrl->n_cand, cap);
    const float t = ctrl->t_final;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long idx = warp; idx < n; idx += nwarps) {
        const Cand e = cand[idx];
        if (!(e.s <= t)) continue;
        int r0[kCells], r1[kCells];
        warp_table(pl, e.i, e.j, e.k, r0, r1);
        if (lane == 0) {
            const double s = k2_f64(r0, r1, k2.lf64);
            const unsigned pos = atomicAdd(&ctrl->n_final, 1u);
            if (pos < (unsigned)kFinalCap) fin[pos] = Final{s, pack_key(e.i, e.j, e.k)};
            else atomicOr(&ctrl->status, kStFinalOverflow);
        }
    }
}

__device__ __forceinline__ bool fin_less(const Final& a, const Final& b) {
    return a.s < b.s || (a.s == b.s && a.key < b.key);
}

__global__ void __launch_bounds__(kFinThreads)
final_kernel(Ctrl* ctrl, const Final* __restrict__ fin, int top_k, double* out_scores,
             int* out_trip) {
    extern __shared__ Final sf[];
    const int tid = threadIdx.x;
    const int n = (int)min(ctrl->n_final, (unsigned)kFinalCap);
    int size = 64;
    while (size < n) size <<= 1;
    for (int idx = tid; idx < size; idx += kFinThreads)
        sf[idx] = (idx < n) ? fin[idx] : Final{__longlong_as_double(0x7ff0000000000000LL), ~0ULL};
    __syncthreads();
    for (int sz = 2; sz <= size; sz <<= 1) {
        for (int stride = sz >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < size / 2; t += kFinThreads) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & sz) == 0);
                const Final a = sf[lo], b = sf[hi];
                if (fin_less(b, a) == up) {
                    sf[lo] = b;
                    sf[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    const int nout = min(top_k, n);
    for (int r = tid; r < nout; r += kFinThreads) {
        const Final e = sf[r];
        out_scores[r] = e.s;
        out_trip[3 * r + 0] = (int)(e.key >> 42);
        out_trip[3 * r + 1] = (int)((e.key >> 21) & 0x1fffffULL);
        out_trip[3 * r + 2] = (int)(e.key & 0x1fffffULL);
    }
    if (tid == 0) {
        ctrl->n_out = (unsigned)nout;
        if (n < top_k) atomicOr(&ctrl->status, kStInternal);
    }
}

__global__ void __launch_bounds__(256)
tables_kernel(Planes pl, PairTables ptab, K2Tables k2, int use_k2, long long n, const int* __restrict__ trip,
              int* __restrict__ out_counts, float* __restrict__ out_s32, double* __restrict__ out_s64,
              Ctrl* ctrl) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = warp; t < n; t += nwarps) {
        const int x = trip[3 * t], y = trip[3 * t + 1], z = trip[3 * t + 2];
        if (x < 0 || y < 0 || z < 0 || x >= pl.M || y >= pl.M || z >= pl.M ||
            (ptab.pt && (x == y || y == z || x == z))) {
            if (lane == 0) atomicOr(&ctrl->status, kStBadIndex);
            continue;
        }
        int r0[kCells], r1[kCells];
        if (ptab.pt) warp_table8(pl, ptab, x, y, z, r0, r1);
        else warp_table(pl, x, y, z, r0, r1);
        if (out_counts && lane < kCells) {
            int v0 = 0, v1 = 0;
#pragma unroll
            for (int q = 0; q < kCells; ++q)
                if (q == lane) {
                    v0 = r0[q];
                    v1 = r1[q];
                }
            out_counts[t * 54 + lane] = v0;
            out_counts[t * 54 + kCells + lane] = v1;
        }
        if (use_k2 && lane == 0) {
            if (out_s32) out_s32[t] = k2_f32(r0, r1, k2.lf2);
            if (out_s64) out_s64[t] = k2_f64(r0, r1, k2.lf64);
        }
    }
}

}  // namespace

cudaError_t launch_reset(Ctrl* ctrl, cudaStream_t st) {
    reset_kernel<<<1, 1, 0, st>>>(ctrl);
    return cudaGetLastError();
}

// Largest error of the products (n + 1/2) * lg2_hw(n + 1) of the K2 bound over every n the scan
// can pass (0 .. N+1): the hardware log against FP64 log2, scaled by the exact multiplier.
__global__ void approx_error_kernel(const double* __restrict__ lf64, int n,
                                    unsigned long long* __restrict__ out) {
    (void)lf64;
    double e = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const float x = exact_float(t);
        const double err = (double)lg2_hw(__fadd_rn(x, 1.f)) - log2((double)t + 1.0);
        e = fmax(e, ((double)t + 0.5) * fabs(err));
    }
    // non-negative doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(e));
}

cudaError_t launch_approx_error(const double* lf64, int n_lf, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int blocks = (n_lf + 255) / 256 < 1024 ? (n_lf + 255) / 256 : 1024;
    approx_error_kernel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(
        lf64, n_lf, reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

cudaError_t launch_select(Ctrl* ctrl, const Cand* cand, long long cap, int top_k, float rel,
                          float abs_, cudaStream_t st) {
    select_kernel<<<1, kSelThreads, 0, st>>>(ctrl, cand, cap, top_k, rel, abs_);
    return cudaGetLastError();
}

cudaError_t launch_rescore(const Planes& pl, const K2Tables& k2, Ctrl* ctrl, const Cand* cand,
                           long long cap, Final* fin, int grid, cudaStream_t st) {
    rescore_kernel<<<grid, 256, 0, st>>>(pl, k2, ctrl, cand, cap, fin);
    return cudaGetLastError();
}

cudaError_t launch_final(Ctrl* ctrl, const Final* fin, int top_k, double* out_scores,
                         int* out_trip, cudaStream_t st) {
    const size_t smem = (size_t)kFinalCap * sizeof(Final);
    cudaError_t e = cudaFuncSetAttribute(final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    final_kernel<<<1, kFinThreads, smem, st>>>(ctrl, fin, top_k, out_scores, out_trip);
    return cudaGetLastError();
}

cudaError_t launch_tables(const Planes& pl, const PairTables* pt, const K2Tables* k2, long long n,
                          const int* trip, int* out_counts, float* out_s32, double* out_s64,
                          Ctrl* ctrl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 7) / 8;  // 8 warps per block
    if (blocks > 65536) blocks = 65536;
    K2Tables kt = k2 ? *k2 : K2Tables{};
    PairTables ptt = pt ? *pt : PairTables{};
    tables_kernel<<<(int)blocks, 256, 0, st>>>(pl, ptt, kt, k2 ? 1 : 0, n, trip, out_counts,
                                               out_s32, out_s64, ctrl);
    return cudaGetLastError();
}

}  // namespace epi3
