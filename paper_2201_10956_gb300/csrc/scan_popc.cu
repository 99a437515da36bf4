// Counting scans: LOP3 AND + POPC over bit planes, fused FP32 K2 and candidate selection
// (Sec. III, Alg. 2, Sec. IV-B), in the paper's 27-cell form and in an 8-cell form.
//
// Work decomposition (GB300 design, not the paper's thread grid): a persistent grid of
// CTAs pulls SNP pairs (i, j) from a global counter, heaviest pairs first (pair index
// p = j (j-1)/2 + i, so k ranges over j+1..M-1).  For its pair a CTA stages the nine
// pair products X[gX] & Y[gY] of both classes in shared memory once (genotype 2 by NOR,
// Sec. IV-A); then each thread owns one third SNP k, streams Z's two planes with
// coalesced 128-bit loads (planes are laid out [class][plane][128-sample group][SNP],
// so consecutive threads read consecutive 16-byte words) and keeps the 54 counts in
// registers, like the private frequency table of Alg. 2.  Pad bits of the last group
// read as genotype 2 in all three SNPs and are removed from cell 26.
//
// Each table is scored in FP32 (k2_f32) and compared with the running threshold.
// Survivors go to a per-CTA shared buffer; when it fills, the CTA sorts it, takes its
// local k-th best s_k, and publishes band_threshold(s_k) with atomicMin: any CTA's
// local k-th best bounds the global one from above, so the shared threshold never
// excludes a triplet that can reach the answer.  At the end each CTA flushes its
// survivors to the global candidate list.
#include "epi3_internal.cuh"

namespace epi3 {

namespace {

__device__ __forceinline__ int popc4(uint4 a, uint4 b) {
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

__device__ __forceinline__ uint4 nor4(uint4 a, uint4 b) {
    return make_uint4(~(a.x | b.x), ~(a.y | b.y), ~(a.z | b.z), ~(a.w | b.w));
}

__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
    return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

// Pair products of class c for SNPs (i, j): sxy[(3 gX + gY) * W4 + w4].
__device__ __forceinline__ void stage_pair(const Planes& pl, int c, int i, int j, uint4* sxy) {
    const int W4 = pl.W4[c];
    const uint4* base = pl.planes + pl.coff[c];
    const size_t pstride = (size_t)W4 * pl.M;
    for (int w4 = threadIdx.x; w4 < W4; w4 += blockDim.x) {
        const size_t o = (size_t)w4 * pl.M;
        const uint4 x0 = __ldg(base + o + i), x1 = __ldg(base + pstride + o + i);
        const uint4 y0 = __ldg(base + o + j), y1 = __ldg(base + pstride + o + j);
        const uint4 x2 = nor4(x0, x1), y2 = nor4(y0, y1);
        const uint4 xs[3] = {x0, x1, x2};
        const uint4 ys[3] = {y0, y1, y2};
#pragma unroll
        for (int gx = 0; gx < 3; ++gx)
#pragma unroll
            for (int gy = 0; gy < 3; ++gy) sxy[(3 * gx + gy) * W4 + w4] = and4(xs[gx], ys[gy]);
    }
}

// 27 counts of class c for third SNP k against the staged pair products.
__device__ __forceinline__ void count_class(const Planes& pl, int c, int k, const uint4* sxy,
                                            int* r) {
    const int W4 = pl.W4[c];
#pragma unroll
    for (int q = 0; q < kCells; ++q) r[q] = 0;
    const uint4* z0p = pl.planes + pl.coff[c] + k;
    const uint4* z1p = z0p + (size_t)W4 * pl.M;
    const size_t M = (size_t)pl.M;
#pragma unroll 1
    for (int w4 = 0; w4 < W4; ++w4) {
        const uint4 z0 = __ldg(z0p + (size_t)w4 * M);
        const uint4 z1 = __ldg(z1p + (size_t)w4 * M);
        const uint4 z2 = nor4(z0, z1);
#pragma unroll
        for (int g = 0; g < 9; ++g) {
            const uint4 v = sxy[g * W4 + w4];
            r[3 * g + 0] += popc4(v, z0);
            r[3 * g + 1] += popc4(v, z1);
            r[3 * g + 2] += popc4(v, z2);
        }
    }
    r[kCells - 1] -= pl.pad[c];
}

// 8-cell form: pair products X[a] & Y[b] for a, b in {0, 1} only: sxy[(2a + b) * W4 + w4].
__device__ __forceinline__ void stage_pair8(const Planes& pl, int c, int i, int j, uint4* sxy) {
    const int W4 = pl.W4[c];
    const uint4* base = pl.planes + pl.coff[c];
    const size_t pstride = (size_t)W4 * pl.M;
    for (int w4 = threadIdx.x; w4 < W4; w4 += blockDim.x) {
        const size_t o = (size_t)w4 * pl.M;
        const uint4 x0 = __ldg(base + o + i), x1 = __ldg(base + pstride + o + i);
        const uint4 y0 = __ldg(base + o + j), y1 = __ldg(base + pstride + o + j);
        sxy[0 * W4 + w4] = and4(x0, y0);
        sxy[1 * W4 + w4] = and4(x0, y1);
        sxy[2 * W4 + w4] = and4(x1, y0);
        sxy[3 * W4 + w4] = and4(x1, y1);
    }
}

// 8 counts n8[4a + 2b + z] of class c for third SNP k (genotypes 0 and 1 only; no pad
// correction: pad bits are 0 in planes 0 and 1).
__device__ __forceinline__ void count_class8(const Planes& pl, int c, int k, const uint4* sxy,
                                             int* n8) {
    const int W4 = pl.W4[c];
#pragma unroll
    for (int q = 0; q < 8; ++q) n8[q] = 0;
    const uint4* z0p = pl.planes + pl.coff[c] + k;
    const uint4* z1p = z0p + (size_t)W4 * pl.M;
    const size_t M = (size_t)pl.M;
#pragma unroll 2
    for (int w4 = 0; w4 < W4; ++w4) {
        const uint4 z0 = __ldg(z0p + (size_t)w4 * M);
        const uint4 z1 = __ldg(z1p + (size_t)w4 * M);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint4 v = sxy[g * W4 + w4];
            n8[2 * g + 0] += popc4(v, z0);
            n8[2 * g + 1] += popc4(v, z1);
        }
    }
}

// Ascending bitonic sort of the kCtaCand shared candidates by FP32 score.
__device__ void sort_cands(Cand* buf) {
    for (int size = 2; size <= kCtaCand; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kCtaCand / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const Cand a = buf[lo], b = buf[hi];
                if ((a.s > b.s) == up) {
                    buf[lo] = b;
                    buf[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

__device__ void flush_cands(const ScanArgs& a, const Cand* buf, int n, float t) {
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const Cand e = buf[idx];
        if (e.s <= t) {
            const unsigned pos = atomicAdd(&a.ctrl->n_cand, 1u);
            if (pos < (unsigned long long)a.cand_cap) a.cand[pos] = e;
            else atomicOr(&a.ctrl->status, kStCandOverflow);
        }
    }
}

// kEight = false: the paper's 27-cell count (Alg. 2 with the pair products staged);
// kEight = true: the 8 cells with genotypes in {0,1} counted, the other 19 derived exactly
// from the pair tables (derive27).  kSum: the instantiation that also adds every table to the
// checksum slots a.tsum (epi3_scan_checksum), kept apart so the product kernel carries no hook.
template <bool kEight, bool kSum>
__global__ void __launch_bounds__(256)
scan_popc_kernel(const ScanArgs a) {
    constexpr int kProd = kEight ? 4 : 9;
    extern __shared__ uint4 sxy[];  // [class][kProd][W4[class]]
    __shared__ Cand cbuf[kCtaCand];
    __shared__ int s_cnt, s_keep;
    __shared__ float s_tloc, s_tglob;
    __shared__ long long s_pair;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M = a.pl.M;
    uint4* sxy0 = sxy;
    uint4* sxy1 = sxy + kProd * a.pl.W4[0];
    __shared__ int4 s_pxy[2];
    __shared__ int2 s_mx[2], s_my[2];
    const float kInf = __int_as_float(0x7f800000);
    if (tid == 0) {
        s_cnt = 0;
        s_tloc = kInf;
    }
    int cnt = 0;  // == s_cnt, kept uniform in registers
    unsigned long long sum_h = 0, sum_n = 0;  // table checksum of this thread (kSum)
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_pair = a.pair_begin + (long long)atomicAdd(&a.ctrl->work, 1ULL);
            s_tglob = __uint_as_float(*(volatile unsigned*)&a.ctrl->thr);
        }
        __syncthreads();
        const long long p = s_pair;
        if (p >= a.pair_end) break;
        int i, j;
        decode_pair(p, &i, &j);
        if (kEight) {
            stage_pair8(a.pl, 0, i, j, sxy0);
            stage_pair8(a.pl, 1, i, j, sxy1);
            if (tid < 2) {
                s_pxy[tid] = __ldg(a.pt.pt + tid * a.pt.n_pairs + pair_index(i, j));
                s_mx[tid] = __ldg(a.pt.marg + (size_t)tid * M + i);
                s_my[tid] = __ldg(a.pt.marg + (size_t)tid * M + j);
            }
        } else {
            stage_pair(a.pl, 0, i, j, sxy0);
            stage_pair(a.pl, 1, i, j, sxy1);
        }
        __syncthreads();
        for (int kb = j + 1; kb < M; kb += nt) {
            const int k = kb + tid;
            bool app = false;
            if (k < M) {
                int r0[kCells], r1[kCells];
                if (kEight) {
                    int n8[8];
                    count_class8(a.pl, 0, k, sxy0, n8);
                    derive27(n8, s_pxy[0], __ldg(a.pt.pt + pair_index(i, k)),
                             __ldg(a.pt.pt + pair_index(j, k)), s_mx[0], s_my[0],
                             __ldg(a.pt.marg + k), a.pt.n_c[0], r0);
                    count_class8(a.pl, 1, k, sxy1, n8);
                    derive27(n8, s_pxy[1], __ldg(a.pt.pt + a.pt.n_pairs + pair_index(i, k)),
                             __ldg(a.pt.pt + a.pt.n_pairs + pair_index(j, k)), s_mx[1], s_my[1],
                             __ldg(a.pt.marg + M + k), a.pt.n_c[1], r1);
                } else {
                    count_class(a.pl, 0, k, sxy0, r0);
                    count_class(a.pl, 1, k, sxy1, r1);
                }
                const float s = k2_f32(r0, r1, a.k2.lf2);
                if (a.dbg) a.dbg[((size_t)i * M + j) * M + k] = s;
                if (kSum) {
                    sum_h += table_hash(i, j, k, r0, r1);
                    ++sum_n;
                }
                if (s <= fminf(s_tloc, s_tglob)) {
                    const int idx = atomicAdd(&s_cnt, 1);
                    cbuf[idx] = Cand{s, i, j, k};
                    app = true;
                }
            }
            cnt += __syncthreads_count(app);
            if (cnt > kCtaCand - nt) {
                // prune: sort, publish the local band threshold, keep what lies inside it
                for (int idx = cnt + tid; idx < kCtaCand; idx += nt) cbuf[idx].s = kInf;
                if (tid == 0) s_keep = 0;
                __syncthreads();
                sort_cands(cbuf);
                if (tid == 0) {
                    const float tl = band_threshold(cbuf[a.top_k - 1].s, a.k2.rel, a.k2.abs_);
                    atomicMin(&a.ctrl->thr, __float_as_uint(tl));
                    s_tloc = fminf(s_tloc, tl);
                    s_tglob = __uint_as_float(*(volatile unsigned*)&a.ctrl->thr);
                }
                __syncthreads();
                const float t = fminf(s_tloc, s_tglob);
                int keep = 0;  // sorted ascending: the kept entries are [0, kept)
                for (int idx = tid; idx < cnt; idx += nt) keep += (cbuf[idx].s <= t);
                if (keep) atomicAdd(&s_keep, keep);
                __syncthreads();
                cnt = s_keep;
                if (cnt > kCtaCand - nt) {
                    flush_cands(a, cbuf, cnt, t);
                    cnt = 0;
                }
                __syncthreads();
                if (tid == 0) s_cnt = cnt;
            }
        }
    }
    // Before the final flush, cut the buffer to this CTA's own band: a CTA that never
    // filled its buffer would otherwise flush every triplet it scored.
    if (cnt >= a.top_k) {
        for (int idx = cnt + tid; idx < kCtaCand; idx += nt) cbuf[idx].s = kInf;
        __syncthreads();
        sort_cands(cbuf);
        if (tid == 0) {
            const float tl = band_threshold(cbuf[a.top_k - 1].s, a.k2.rel, a.k2.abs_);
            atomicMin(&a.ctrl->thr, __float_as_uint(tl));
            s_tloc = fminf(s_tloc, tl);
        }
    }
    __syncthreads();
    const float t = fminf(s_tloc, __uint_as_float(*(volatile unsigned*)&a.ctrl->thr));
    flush_cands(a, cbuf, cnt, t);
    if (kSum) table_sum_flush(a.tsum, sum_h, sum_n);
}

}  // namespace

size_t scan_popc_smem(const Planes& pl) {
    return (size_t)9 * (pl.W4[0] + pl.W4[1]) * sizeof(uint4);
}

size_t scan_popc8_smem(const Planes& pl) {
    return (size_t)4 * (pl.W4[0] + pl.W4[1]) * sizeof(uint4);
}

// The dynamic shared-memory cap is a per-kernel attribute: set it to the largest size any
// data set can need (not to this one's), so launches of several data sets (a batch graph)
// all stay within it.
constexpr int kPopcSmemCap = 200 * 1024;

template <bool kEight>
static cudaError_t occupancy(int block, size_t smem, int* ctas_per_sm) {
    if (smem > (size_t)kPopcSmemCap) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(scan_popc_kernel<kEight, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPopcSmemCap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(scan_popc_kernel<kEight, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPopcSmemCap);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,
                                                         scan_popc_kernel<kEight, false>, block, smem);
}

cudaError_t scan_popc_occupancy(int block, size_t smem, int* ctas_per_sm) {
    return occupancy<false>(block, smem, ctas_per_sm);
}

cudaError_t scan_popc8_occupancy(int block, size_t smem, int* ctas_per_sm) {
    return occupancy<true>(block, smem, ctas_per_sm);
}

cudaError_t launch_scan_popc(const ScanArgs& a, int grid, int block, size_t smem,
                             cudaStream_t st) {
    if (a.tsum) scan_popc_kernel<false, true><<<grid, block, smem, st>>>(a);
    else scan_popc_kernel<false, false><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan_popc8(const ScanArgs& a, int grid, int block, size_t smem,
                              cudaStream_t st) {
    if (a.tsum) scan_popc_kernel<true, true><<<grid, block, smem, st>>>(a);
    else scan_popc_kernel<true, false><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace epi3
