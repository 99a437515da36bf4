// Tensor-core counting scan on sample-compacted operands (path EPI3_PATH_MMA4C).
//
// For a fixed first SNP i, class c and genotype a of SNP i, let S be the samples of class c
// with g_i = a.  The cells (a, b, z) with b, z in {0,1} of every triplet (i, j, k) are
//     n(a, b, z) = sum over s in S of [g_j(s) = b] [g_k(s) = z],
// a plain GEMM of two one-hot matrices over the samples of S: rows (j, b) x columns (k, z).  Two
// genotypes a of SNP i are counted this way, the two least frequent over all samples; the most
// frequent one is derived with the other 19 cells (the same genotype in both classes), so the
// GEMMs run over the smallest share of the samples.  The samples of each of the four sets
// (c, a) are gathered once per first SNP ("compaction": bit extraction from the packed planes,
// expansion to FP4 E2M1 0/1 values in the 128B-swizzled shared-memory image), and the scan
// multiplies compacted chunks straight from L2: both MMA operands come from shared memory,
// filled by bulk copies, with no operand formed on chip and 4 MACs per sample-triplet whose
// first-SNP genotype is counted.  The epilogue relabels SNP i's genotypes (counted ones 0 and 1,
// the derived one 2) in its pair-table and marginal inputs, derives the 19 other cells from pair
// tables and marginals, and restores the genotype order before the exact table is scored: K2
// and the candidate band exactly as in the other scans (Eq. 1; the paper counts with POPCNT,
// Sec. IV, and points at tensor-core formulations in Sec. II).
//
// Every set carries one bias sample (a 1 in every row) after its samples, so every accumulator
// ends at count + 1, the argument of the epilogue's count + 1 arithmetic.
//
// Tile = (i, 64 second SNPs j, 32 third SNPs k): MMA M = 128 rows (j, b), N = 64 columns (k, z),
// kind::mxf4 (K = 64 FP4 samples per instruction, four per 256-sample step, every block scale
// 2^0), FP32 accumulation in tensor memory: one 64-column region per set, regions taken from a
// ring of seven so that the next tile's first sets run while the epilogue reads this one.
// Shared memory: a ring of three slots of two K-steps each (A 32 KB in one copy, B 2 x 8 KB),
// with one full barrier, one empty barrier and one tcgen05.commit per slot (a set's odd last
// step takes half a slot): every commit costs the tensor pipe a bubble, so fewer, larger slots
// beat one slot per step.
//
// Warp roles (16 warps): 0 = operand loader + tensor-memory allocator, 1 = MMA issuer (both as
// whole warps, one elected lane issuing), 2-3 idle, 4-15 = epilogue (three warps per
// tensor-memory lane quadrant); registers move from the first warp group to the epilogue
// (setmaxnreg).  Every mbarrier wait is bounded; on timeout the kernel
// records kStTimeout, waits for its own copies and MMAs, frees tensor memory and returns.
#include <algorithm>
#include <atomic>

#include "epi3_internal.cuh"
#include "tc_common.cuh"
#include "bit_compress.cuh"

namespace epi3 {

namespace {

constexpr int kCmpChunk = 16384;         // one compacted chunk: 128 rows (m, z) x 256 samples
constexpr int kMaskWords = 128;          // selection words staged per pass of the compaction
constexpr int kSlabBytes = 32 * 128;     // one warp's 32 rows of a chunk: 4 KB, contiguous

}  // namespace

namespace {

// One compacted output stream of a thread: 32-bit words of compacted samples, written one at
// a time as 16 E2M1 bytes into unit (word % 8) of the thread's row in step (word / 8).
struct CmpStream {
    unsigned long long acc;     // pending bits, low first
    int fill;                   // pending bit count
    int word;                   // words written
};

// A word goes to the warp's shared-memory image of its 32 rows of the current chunk (the same
// 128B-swizzled layout); when the K-step's eighth word is in, the warp writes the 4 KB slab out
// with contiguous 16-byte stores (every thread of the CTA emits at the same points: the bit
// counts per word are the CTA's).
__device__ __forceinline__ void cmp_emit(uint8_t* set_base, uint8_t* slab, int row, CmpStream& st,
                                         uint32_t w) {
    uint4 v;
    v.x = byte_to_e2m1(w);
    v.y = byte_to_e2m1(w >> 8);
    v.z = byte_to_e2m1(w >> 16);
    v.w = byte_to_e2m1(w >> 24);
    const uint32_t u = (uint32_t)(st.word & 7);
    *reinterpret_cast<uint4*>(slab + sw128_off((uint32_t)(row & 31), u)) = v;
    if (u == 7) {  // uniform across the warp
        __syncwarp();
        uint8_t* const dst = set_base + (size_t)(st.word >> 3) * kCmpChunk + (size_t)(row & ~31) * 128;
        const int lane = row & 31;
#pragma unroll
        for (int j = 0; j < kSlabBytes / 512; ++j) {
            const int off = 16 * (lane + 32 * j);
            *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(slab + off);
        }
        __syncwarp();
    }
    ++st.word;
}

__device__ __forceinline__ void cmp_push(uint8_t* set_base, uint8_t* slab, int row, CmpStream& st,
                                         uint32_t bits, int n) {
    st.acc |= (unsigned long long)bits << st.fill;
    st.fill += n;
    if (st.fill >= 32) {
        cmp_emit(set_base, slab, row, st, (uint32_t)st.acc);
        st.acc >>= 32;
        st.fill -= 32;
    }
}

constexpr int kCompactThreads = 128;     // one row (SNP, genotype) of the 64-SNP block per thread

// Push the bits of one 32-sample word selected by a set's mask: compress by the mask (Hacker's
// Delight 7-4, masks prepared once per word by cmp_masks), append to the stream, emit each full
// word.
__device__ __forceinline__ void cmp_word(uint8_t* set_base, uint8_t* slab, int row, CmpStream& st,
                                         uint32_t x, uint32_t mask, const uint32_t* mv, int n) {
    if (n == 0) return;
    cmp_push(set_base, slab, row, st, n == 32 ? x : cmp_bits(x, mask, mv), n);
}

// One selection word's masks for both sets, read with four 16-byte shared-memory loads:
// {mask0, mask1, pop0, pop1}, mv0[0..3], mv1[0..3], {mv0[4], mv1[4], -, -}.
struct MaskWord {
    uint4 q[4];
};

// Rows of a chunk come in 16-row groups: row 16 G + 8 z + r holds SNP m = 64 b + 8 G + r with
// genotype z (8 SNPs of genotype 0, then the same 8 of genotype 1), so that a 16x256b
// tensor-memory load hands a thread both genotype rows of one SNP (see the epilogue).
// CTA (b, i - i0, c), 128 threads: thread r writes row r of every chunk of block b for the two
// sets (c, 0) and (c, 1) of first SNP i: the bits [g_m = z] of the class-c samples whose g_i is
// the set's counted genotype, in sample order, then the bias sample, then zeros to the set's
// K-steps.
// Plane words come four at a time (one 16-byte load per 128 samples, the next one in flight
// while the current one is compressed); each word's masks of both sets come in four 16-byte
// shared-memory loads.
__global__ void __launch_bounds__(kCompactThreads)
compact_kernel(Planes pl, const CmpFirst* __restrict__ firsts, int i0, uint8_t* __restrict__ cmp) {
    __shared__ MaskWord s_w[kMaskWords];
    __shared__ __align__(128) uint8_t s_slab[2][kCompactThreads / 32][kSlabBytes];
    const int b = blockIdx.x, i = i0 + (int)blockIdx.y, c = (int)blockIdx.z;
    // the fields this CTA needs, read in place (a local copy indexed by the class would live in
    // local memory)
    const CmpFirst* const fp = firsts + blockIdx.y;
    const int b_lo = fp->b_lo;
    if (b < b_lo) return;  // whole CTA: no block before the first SNP's successors
    const int ks0 = fp->ks[2 * c], ks1 = fp->ks[2 * c + 1];
    const long long fb0 = fp->base[2 * c], fb1 = fp->base[2 * c + 1];
    const int drop = fp->drop;
    const int M = pl.M;
    const int r = threadIdx.x, z = (r >> 3) & 1;
    const int m = 64 * b + 8 * (r >> 4) + (r & 7);
    const long long coff = c ? pl.coff[1] : pl.coff[0];
    const int W4 = c ? pl.W4[1] : pl.W4[0];
    const int W = 4 * W4;                       // 32-sample words of the class
    const int Nc = 128 * W4 - (c ? pl.pad[1] : pl.pad[0]);
    uint8_t* const base0 = cmp + (size_t)(fb0 + (long long)(b - b_lo) * ks0) * kCmpChunk;
    uint8_t* const base1 = cmp + (size_t)(fb1 + (long long)(b - b_lo) * ks1) * kCmpChunk;
    CmpStream s0{0ull, 0, 0}, s1{0ull, 0, 0};   // sets (c, 0) and (c, 1)
    uint8_t* const slab0 = s_slab[0][r >> 5];
    uint8_t* const slab1 = s_slab[1][r >> 5];
    const uint4* const pc = pl.planes + coff;   // [plane][group][SNP] of 4 words
    const uint32_t* const prow = reinterpret_cast<const uint32_t*>(pc);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (int w0 = 0; w0 < W; w0 += kMaskWords) {
        const int nw = min(kMaskWords, W - w0);   // a multiple of 4
        __syncthreads();  // the previous pass's masks are no longer read
        for (int w = threadIdx.x; w < nw; w += blockDim.x) {
            // word w0 + w of planes 0 and 1 of SNP i: group (w0 + w) / 4, word (w0 + w) % 4
            const int ww = w0 + w;
            const uint32_t g0 = prow[((size_t)(ww >> 2) * M + i) * 4 + (ww & 3)];
            const uint32_t g1 = prow[((size_t)(W4 + (ww >> 2)) * M + i) * 4 + (ww & 3)];
            // genotype 2 by NOR, without the pad positions past the class's last sample
            const int nv = Nc - 32 * ww;
            const uint32_t valid = nv >= 32 ? 0xFFFFFFFFu : (nv <= 0 ? 0u : (1u << nv) - 1u);
            const uint32_t g2 = ~(g0 | g1) & valid;
            // the two counted genotypes, ascending (cmp_geno)
            const uint32_t mk0 = drop == 0 ? g1 : g0;
            const uint32_t mk1 = drop == 2 ? g1 : g2;
            uint32_t v0[5], v1[5];
            cmp_masks(mk0, v0);
            cmp_masks(mk1, v1);
            MaskWord e;
            e.q[0] = make_uint4(mk0, mk1, (uint32_t)__popc(mk0), (uint32_t)__popc(mk1));
            e.q[1] = make_uint4(v0[0], v0[1], v0[2], v0[3]);
            e.q[2] = make_uint4(v1[0], v1[1], v1[2], v1[3]);
            e.q[3] = make_uint4(v0[4], v1[4], 0u, 0u);
            s_w[w] = e;
        }
        __syncthreads();
        const int g0 = w0 >> 2, ng = nw >> 2;
        const uint4* const src = pc + (size_t)(z * W4 + g0) * M + m;   // this row's plane
        uint4 vn = m < M ? __ldg(src) : zero4;
        for (int g = 0; g < ng; ++g) {
            const uint4 v = vn;
            if (g + 1 < ng) vn = m < M ? __ldg(src + (size_t)(g + 1) * M) : zero4;
            const uint32_t xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const MaskWord& mw = s_w[4 * g + e];
                const uint4 h = mw.q[0], a0 = mw.q[1], a1 = mw.q[2], a4 = mw.q[3];
                const uint32_t mv0[5] = {a0.x, a0.y, a0.z, a0.w, a4.x};
                const uint32_t mv1[5] = {a1.x, a1.y, a1.z, a1.w, a4.y};
                cmp_word(base0, slab0, r, s0, xs[e], h.x, mv0, (int)h.z);
                cmp_word(base1, slab1, r, s1, xs[e], h.y, mv1, (int)h.w);
            }
        }
    }
    // the bias sample, then zeros up to the set's K-steps (8 words each)
    cmp_push(base0, slab0, r, s0, 1u, 1);
    cmp_push(base1, slab1, r, s1, 1u, 1);
    for (const int words = 8 * ks0; s0.word < words;) {
        cmp_emit(base0, slab0, r, s0, (uint32_t)s0.acc);
        s0.acc >>= 32;
    }
    for (const int words = 8 * ks1; s1.word < words;) {
        cmp_emit(base1, slab1, r, s1, (uint32_t)s1.acc);
        s1.acc >>= 32;
    }
}

// ------------------------------------------------------------------ the scan kernel
constexpr int kTJ = 64;                  // second SNPs per tile: A rows (j, b)
constexpr int kTK = 32;                  // third SNPs per tile: B rows (k, z), MMA N = 64
constexpr int kN = 2 * kTK;
constexpr int kSlotSteps = 2;            // K-steps per shared-memory slot: one commit frees both
constexpr int kSlots = 3;                // shared-memory ring
constexpr int kStepA = kCmpChunk;        // one K-step of A: 128 rows x 128 B
constexpr int kStepB = kCmpChunk / 2;    // one K-step of B: 64 rows x 128 B
constexpr int kSlotA = kSlotSteps * kStepA;
constexpr int kSlotB = kSlotSteps * kStepB;
constexpr int kCmpRegions = 7;           // 64-column accumulator regions (columns 0..447)
constexpr uint32_t kCmpSfCol = 480;      // block scales: A at 480..495, B at 496..511
constexpr int kCmpThreads = 512;
constexpr int kCmpEpiWarp0 = 4, kCmpEpiWarps = 12, kCmpEpiThreads = kCmpEpiWarps * 32;
constexpr int kCmpEpiParts = kCmpEpiWarps / 4;   // epilogue warps per tensor-memory lane quadrant
// the epilogue's items: per quadrant 2 lane groups (8 second SNPs each) x 4 column groups (8 third
// SNPs each), split 3 / 3 / 2 over its three warps
static_assert(kCmpEpiParts == 3 && kTJ == 4 * 2 * 8 && kTK == 4 * 8, "epilogue item split");
constexpr int kCmpRegLaunch = 128, kCmpRegCtl = 56, kCmpRegEpi = 152;
static_assert(kCmpRegCtl + 3 * kCmpRegEpi == 4 * kCmpRegLaunch, "register split");
static_assert(kCmpThreads * kCmpRegLaunch == 65536, "the launch holds the whole register file");
static_assert(kCmpRegions * kN <= (int)kCmpSfCol, "tensor memory budget");

// Instruction descriptor of kind::mxf4: A/B E2M1, UE8M0 scales, K-major, N = 64, M = 128.
constexpr uint32_t kIdescCmp = (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | (1u << 23) |
                               ((128u >> 4) << 24);

// Issued warp-wide: elect.sync picks the lane that issues (see tc_common.cuh).
__device__ __forceinline__ void mma_ss_mx_elect(uint32_t d, uint64_t a, uint64_t b, uint32_t acc,
                                                uint32_t sfa, uint32_t sfb) {
    asm volatile(
        "{\n .reg .pred p, e;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %3, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %6,"
        " [%4], [%5], p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(acc), "r"(sfa), "r"(sfb), "r"(kIdescCmp) : "memory");
}

// 16 lanes x 16 FP32 columns from taddr: thread t gets lane t / 4 (v[0..1]) and lane t / 4 + 8
// (v[2..3]) at columns 2 (t % 4) + {0, 1}, then the same at columns + 8 (v[4..7]).
__device__ __forceinline__ void tc_ld16x2(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7])
        : "r"(taddr));
}

}  // namespace


namespace {

struct CmpTile {
    int f;                       // first SNP, relative to the range
    int jb, kb;                  // 64-SNP block of j, 32-SNP block of k
};

// Tile t of the range: first SNPs in order, then j blocks from b_lo (to jb_end), then k blocks
// from 2 jb.
__device__ __forceinline__ CmpTile cmp_tile(const CmpArgs& a, long long t) {
    int lo = 0, hi = a.n_first;  // last f with tile0 <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.firsts[mid].tile0 <= t) lo = mid;
        else hi = mid;
    }
    CmpTile r;
    r.f = lo;
    long long u = t - a.firsts[lo].tile0;
    const int nk = (a.cd.pl.M + kTK - 1) / kTK;
    int jb = a.firsts[lo].b_lo;
    while (u >= nk - 2 * jb) {
        u -= nk - 2 * jb;
        ++jb;
    }
    r.jb = jb;
    r.kb = 2 * jb + (int)u;
    return r;
}

// kInstr: the instrumented instantiation (table checksums; with a.prof, per role the cycles spent
// waiting, summed over CTAs: [0] loader on free slots, [1] MMA issuer on loaded slots, [2] MMA
// issuer on free accumulator regions, [4] epilogue thread 0 on finished tiles, [5] kernel cycles,
// [7] MMA issuer issuing MMAs and commits).
// kPaired: the epilogue derives the cells and the bound of a lane's two triplets together in
// f32x2 instructions (fewer instructions, more registers live: faster where the MMA pipeline
// bounds the scan, slower where the epilogue does; the tuner measures both).
template <bool kInstr, bool kPaired>
__global__ void __launch_bounds__(kCmpThreads, 1) scan_cmp_kernel(const CmpArgs a) {
    const long long t_start = kInstr ? clock64() : 0;
    unsigned long long* const prof = kInstr ? a.prof : nullptr;
    unsigned long long w_acc = 0, w_acc2 = 0, w_acc3 = 0;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* sA = base;                                 // [kSlots][kSlotSteps][16 KB] rows (j, b)
    uint8_t* sB = base + kSlots * kSlotA;               // [kSlots][kSlotSteps][8 KB] rows (k, z)
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kSlots * kSlotB);
    // bars: fullS[kSlots], emptyS[kSlots], accF[2], regE[kCmpRegions], drain
    constexpr int kNBars = 2 * kSlots + 2 + kCmpRegions + 1;
    static_assert(kNBars * 8 + 8 <= 256, "barrier area");
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile unsigned* loader_steps = reinterpret_cast<volatile unsigned*>(tmem_slot + 2);
    EpiShared& es = *reinterpret_cast<EpiShared*>(reinterpret_cast<uint8_t*>(bars) + 256);
    const uint32_t fullS0 = smem_u32(bars), emptyS0 = smem_u32(bars + kSlots),
                   accF0 = smem_u32(bars + 2 * kSlots), regE0 = accF0 + 16,
                   drain0 = regE0 + 8 * kCmpRegions;
    const CohortDev& cd = a.cd;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(fullS0 + 8 * s, 1);
            mbar_init(emptyS0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) mbar_init(accF0 + 8 * b, 1);
        for (int r = 0; r < kCmpRegions; ++r) mbar_init(regE0 + 8 * r, kCmpEpiWarps);
        mbar_init(drain0, 1);
        *abort_flag = 0;
        *loader_steps = 0u;
        es.cnt = 0;
        es.tloc = __int_as_float(0x7f800000);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp < 4) {  // block scale factors 2^0 (UE8M0 127) in every byte of the scale columns
        uint32_t one[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) one[t] = 0x7F7F7F7Fu;
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
            ::"r"(tmem + ((uint32_t)(32 * warp) << 16) + kCmpSfCol), "r"(one[0]), "r"(one[1]),
              "r"(one[2]), "r"(one[3]), "r"(one[4]), "r"(one[5]), "r"(one[6]), "r"(one[7]),
              "r"(one[8]), "r"(one[9]), "r"(one[10]), "r"(one[11]), "r"(one[12]), "r"(one[13]),
              "r"(one[14]), "r"(one[15]), "r"(one[16]), "r"(one[17]), "r"(one[18]), "r"(one[19]),
              "r"(one[20]), "r"(one[21]), "r"(one[22]), "r"(one[23]), "r"(one[24]), "r"(one[25]),
              "r"(one[26]), "r"(one[27]), "r"(one[28]), "r"(one[29]), "r"(one[30]), "r"(one[31])
            : "memory");
        tc_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const long long my_tiles =
        a.n_tiles > blockIdx.x ? (a.n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    // role: 1 loader (on a free slot), 2 MMA issuer (region), 3 MMA issuer (operands),
    // 4 epilogue (accumulators), 5 the timeout test hook
    auto fail_at = [&](unsigned role, long long tl, int q, int ks, unsigned extra = 0u) {
        *abort_flag = 1;
        if (atomicCAS(&cd.ctrl->wait_role, 0u, role) == 0u) {
            cd.ctrl->wait_tile = (unsigned)tl;
            cd.ctrl->wait_set = (unsigned)q;
            cd.ctrl->wait_step = (unsigned)ks;
            cd.ctrl->pad_[0] = extra;
            cd.ctrl->pad_[1] = *loader_steps;
        }
        atomicOr(&cd.ctrl->status, kStTimeout);
    };

    if (warp < kCmpEpiWarp0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kCmpRegCtl));
        // The loader (warp 0) and the MMA issuer (warp 1) run as whole warps with warp-uniform
        // control flow; one elected lane issues each copy, MMA and commit.  Values read from
        // memory are broadcast from lane 0 so that every operand is provably uniform.
        if (warp == 0) {
            // ------------------------------------------------ operand loader
            Ring rs{0, 0u};
            uint32_t used = 0, fph = 0;
            bool stop = false;
            for (long long tl = 0; tl < my_tiles && !stop; ++tl) {
                const CmpTile T = cmp_tile(a, blockIdx.x + tl * gridDim.x);
                const int f = warp_uniform(T.f), jb = warp_uniform(T.jb), kb = warp_uniform(T.kb);
                const CmpFirst& F = a.firsts[f];
                const int b_lo = warp_uniform(F.b_lo);
                for (int q = 0; q < kCmpSets && !stop; ++q) {
                    const int KS = warp_uniform(F.ks[q]);
                    const long long base_q = warp_uniform(F.base[q]);
                    const long long ca0 = base_q + (long long)(jb - b_lo) * KS;
                    const long long cb0 = base_q + (long long)((kb >> 1) - b_lo) * KS;
                    const size_t boff = (size_t)(kb & 1) * kStepB;
                    for (int ks = 0; ks < KS; ks += kSlotSteps) {
                        // a slot takes up to kSlotSteps consecutive steps of one set: their A
                        // chunks are adjacent (one copy), their B halves are not
                        const int n = min(kSlotSteps, KS - ks);
                        const int s = rs.s;
                        const bool got = mbar_wait_t(emptyS0 + 8 * s, rs.ph ^ 1u, abort_flag,
                                                     (prof && lane == 0) ? &w_acc : nullptr);
                        if (!__all_sync(0xffffffffu, got)) {
                            if (lane == 0) fail_at(1, tl, q, ks, (unsigned)s | (rs.ph << 8));
                            stop = true;
                            break;
                        }
                        const uint32_t fb = fullS0 + 8 * s;
                        mbar_arrive_tx_elect(fb, (unsigned)(n * (kStepA + kStepB)));
                        bulk_g2s_elect(smem_u32(sA + s * kSlotA), a.cmp + (size_t)(ca0 + ks) * kCmpChunk,
                                       (unsigned)(n * kStepA), fb);
                        for (int h = 0; h < n; ++h)
                            bulk_g2s_elect(smem_u32(sB + s * kSlotB + h * kStepB),
                                           a.cmp + (size_t)(cb0 + ks + h) * kCmpChunk + boff, kStepB, fb);
                        used |= 1u << s;
                        fph ^= 1u << s;
                        ring_next(rs, kSlots);
                        if (lane == 0) *loader_steps = *loader_steps + (unsigned)n;
                    }
                }
            }
            // drain: the copies issued must land before the CTA exits
            for (int b = 0; b < kSlots; ++b) {
                if (!((used >> b) & 1u)) continue;
                volatile int no_abort = 0;
                mbar_wait(fullS0 + 8 * b, ((fph >> b) & 1u) ^ 1u, &no_abort);
            }
            __syncwarp();
        } else if (warp == 1) {
            // ------------------------------------------------ MMA issuer
            bool ok = true;
            if (cd.inject_timeout) {  // test hook: a wait that can only run out (about 1 s)
                const bool got = mbar_wait(drain0, 0, abort_flag);
                if (!__all_sync(0xffffffffu, got) && lane == 0) fail_at(5, 0, 0, 0);
                ok = false;
            }
            Ring rR{0, 0u}, rs{0, 0u};
            unsigned consumed = 0;
            const uint32_t aS = smem_u32(sA), bS = smem_u32(sB);
            for (long long tl = 0; tl < my_tiles && ok; ++tl) {
                const CmpTile T = cmp_tile(a, blockIdx.x + tl * gridDim.x);
                const CmpFirst& F = a.firsts[warp_uniform(T.f)];
                for (int q = 0; q < kCmpSets && ok; ++q) {
                    const bool freed = mbar_wait_t(regE0 + 8 * rR.s, rR.ph ^ 1u, abort_flag,
                                                   (prof && lane == 0) ? &w_acc2 : nullptr);
                    if (!__all_sync(0xffffffffu, freed)) {
                        if (lane == 0) fail_at(2, tl, q, 0);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(rR.s * kN);
                    ring_next(rR, kCmpRegions);
                    const int KS = warp_uniform(F.ks[q]);
                    for (int ks = 0; ks < KS; ks += kSlotSteps) {
                        const int n = min(kSlotSteps, KS - ks);
                        const int s = rs.s;
                        const bool got = mbar_wait_t(fullS0 + 8 * s, rs.ph, abort_flag,
                                                     (prof && lane == 0) ? &w_acc : nullptr);
                        if (!__all_sync(0xffffffffu, got)) {
                            if (lane == 0) fail_at(3, tl, q, ks, (unsigned)s | (rs.ph << 8) | (consumed << 16));
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const long long t_issue = prof ? clock64() : 0;
                        for (int h = 0; h < n; ++h) {
                            const uint64_t da = sw128_desc(aS + (uint32_t)(s * kSlotA + h * kStepA));
                            const uint64_t db = sw128_desc(bS + (uint32_t)(s * kSlotB + h * kStepB));
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)  // 32 bytes (64 samples) of K per MMA
                                mma_ss_mx_elect(d, da + 2 * kk, db + 2 * kk, (ks | h | kk) ? 1u : 0u,
                                                tmem + kCmpSfCol, tmem + kCmpSfCol + 16);
                        }
                        tc_commit_elect(emptyS0 + 8 * s);  // the slot is free once these MMAs complete
                        if (prof) w_acc3 += (unsigned long long)(clock64() - t_issue);
                        ring_next(rs, kSlots);
                        consumed += (unsigned)n;
                    }
                }
                if (ok) tc_commit_elect(accF0 + 8 * (int)(tl & 1));
            }
            // every MMA issued must complete before tensor memory is released
            tc_commit_elect(drain0);
            volatile int no_abort = 0;
            mbar_wait(drain0, 0, &no_abort);
            __syncwarp();
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kCmpRegEpi));
        // ------------------------------------------------ epilogue
        // Per set (c, a), tensor-memory lane 16 G + 8 b + r holds the counts + 1 of second SNP
        // jl = 8 G + r with genotype b, in column 16 H + 8 z + s for third SNP kl = 8 H + s with
        // genotype z (the chunks' row order).  A 16x256b.x2 load at lane group G, column group H
        // gives thread t the cells (b, z) of jl = 8 G + t / 4 and kl = 8 H + 2 (t % 4) + e,
        // e = 0, 1, in registers 4 z + 2 b + e: all 8 cells of a set for two triplets.  Items of
        // a quadrant: lane groups G = 2 quad + h (h = 0, 1) x column groups H = 0..3; part 0
        // takes h = 0 with H = 0..2, part 1 h = 1 with H = 0..2, part 2 both h with H = 3.
        const int tid = threadIdx.x - kCmpEpiWarp0 * 32;     // 0 .. 383
        const int quad = warp & 3, part = (warp - kCmpEpiWarp0) >> 2;
        const int trow = lane >> 2, tcol = 2 * (lane & 3);
        const int M = cd.pl.M;
        const PairTables pt = cd.pt;
        const float2* lf2 = cd.k2.lf2;
        const float prune = cd.k2.prune_delta;
        float* dbg = cd.dbg;
        Ctrl* ctrl = cd.ctrl;
        const bool tsum_on = kInstr && cd.tsum != nullptr;
        const bool pruning = !dbg && !tsum_on && prune > 0.f;
        unsigned long long sum_h = 0, sum_n = 0;
        Ring rR{0, 0u};
        for (long long tl = 0; tl < my_tiles; ++tl) {
            const CmpTile T = cmp_tile(a, blockIdx.x + tl * gridDim.x);
            const int i = a.i0 + T.f, kb0 = kTK * T.kb;
            bool bad = false;
            if (tid == 0) {
                bad = !mbar_wait_t(accF0 + 8 * (int)(tl & 1), (unsigned)((tl >> 1) & 1), abort_flag,
                                   prof ? &w_acc : nullptr);
                if (bad) fail_at(4, tl, 0, 0);
            }
            // uniform stop; also orders the previous tile's candidate bookkeeping before this
            // tile's appends, and thread 0's observation of the barrier before every TMEM read
            if (epi_sync_or<kCmpEpiThreads>(bad || *abort_flag)) break;
            tc_fence_after();
            int regs[kCmpSets];
#pragma unroll
            for (int q = 0; q < kCmpSets; ++q) {
                regs[q] = rR.s;
                ring_next(rR, kCmpRegions);
            }
            // the derived first-SNP genotype; the first SNP's inputs relabelled
            const int dsel = __ldg(&a.firsts[T.f].drop);
            int2 mx[2];
            mx[0] = relabel_marg(__ldg(pt.marg + i), pt.n_c[0], dsel);
            mx[1] = relabel_marg(__ldg(pt.marg + M + i), pt.n_c[1], dsel);
            int cur_h = -1, j = 0;
            bool jrow = false;
            RowCells rcl[2];
            const int n_items = part == 2 ? 2 : 3;
            for (int it = 0; it < n_items; ++it) {
                const int h = part == 2 ? it : part, H = part == 2 ? 3 : it;
                if (h != cur_h) {  // this thread's second SNP and its row cells
                    cur_h = h;
                    j = kTJ * T.jb + 8 * (2 * quad + h) + trow;
                    long long pij = -1;
                    if (j < M && j > i) {
                        pij = pair_index(i, j);
                        if (pij < cd.pair_begin || pij >= cd.pair_end) pij = -1;
                    }
                    jrow = pij >= 0;
                    int4 pxy[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
                    int2 my[2] = {make_int2(0, 0), make_int2(0, 0)};
                    if (jrow) {
                        pxy[0] = __ldg(pt.pt + pij);
                        pxy[1] = __ldg(pt.pt + pt.n_pairs + pij);
                        my[0] = __ldg(pt.marg + j);
                        my[1] = __ldg(pt.marg + M + j);
                    }
                    rcl[0] = row_cells(relabel_xy(pxy[0], my[0], dsel), mx[0], my[0], pt.n_c[0]);
                    rcl[1] = row_cells(relabel_xy(pxy[1], my[1], dsel), mx[1], my[1], pt.n_c[1]);
                }
                const float thr_g = __uint_as_float(*(volatile unsigned*)&ctrl->thr);
                // this thread's two triplets: k = kb0 + 8 H + tcol + m; pair-table rows first
                float4 tik[2][2], tjk[2][2];
                float2 tmk[2][2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = kb0 + 8 * H + tcol + m;
                    const bool val = jrow && k > j && k < M;
                    const long long pik = val ? pair_index(i, k) : 0, pjk = val ? pair_index(j, k) : 0;
                    const int kq = val ? k : 0;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        tik[m][c] = __ldg(pt.ptf + c * pt.n_pairs + pik);
                        tjk[m][c] = __ldg(pt.ptf + c * pt.n_pairs + pjk);
                        tmk[m][c] = __ldg(pt.margf + (size_t)c * M + kq);
                    }
                }
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int c = 0; c < 2; ++c) tik[m][c] = relabel_xz(tik[m][c], tmk[m][c], dsel);
                uint32_t v[kCmpSets][8];
#pragma unroll
                for (int q = 0; q < kCmpSets; ++q)
                    tc_ld16x2(tmem + ((uint32_t)(32 * quad + 16 * h) << 16) + (uint32_t)(regs[q] * kN + 16 * H),
                              v[q]);
                tc_wait_ld();
                // n8[c][4 a + 2 b + z] = count + 1 of triplet m: set 2 c + a, register 4 z + 2 b + m
                auto n8_of = [&](int m, int c, int e) {
                    return __uint_as_float(v[2 * c + (e >> 2)][4 * (e & 1) + 2 * ((e >> 1) & 1) + m]);
                };
                // paired form: the lane's two triplets in the two lanes of f32x2 instructions
                // (x: m = 0, y: m = 1); the inputs are gathered into lane pairs once, and the bound
                // derives both classes' cells on the fly
                float2 n8p[2][8], xzp[2][2][2], yzp[2][2][2], mzp[2][2], bnd = make_float2(0.f, 0.f);
                if constexpr (kPaired) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) n8p[c][e] = make_float2(n8_of(0, c, e), n8_of(1, c, e));
                        const float4 x0 = tik[0][c], x1 = tik[1][c], y0 = tjk[0][c], y1 = tjk[1][c];
                        xzp[c][0][0] = make_float2(x0.x, x1.x); xzp[c][0][1] = make_float2(x0.y, x1.y);
                        xzp[c][1][0] = make_float2(x0.z, x1.z); xzp[c][1][1] = make_float2(x0.w, x1.w);
                        yzp[c][0][0] = make_float2(y0.x, y1.x); yzp[c][0][1] = make_float2(y0.y, y1.y);
                        yzp[c][1][0] = make_float2(y0.z, y1.z); yzp[c][1][1] = make_float2(y0.w, y1.w);
                        mzp[c][0] = make_float2(tmk[0][c].x, tmk[1][c].x);
                        mzp[c][1] = make_float2(tmk[0][c].y, tmk[1][c].y);
                    }
                    if (pruning) {
                        const float2 sacc = k2_bound_cells<LaneOps2>(n8p, rcl, xzp, yzp, mzp);
                        bnd = make_float2(k2_bound_finish(sacc.x), k2_bound_finish(sacc.y));
                    }
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = kb0 + 8 * H + tcol + m;
                    if (!(jrow && k > j && k < M)) continue;
                    // triplet m's inputs: counted cells, pair-table rows (X, Z), (Y, Z), marginal of Z
                    float n8[2][8], xz[2][2][2], yz[2][2][2], mz[2][2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if constexpr (kPaired) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) n8[c][e] = m ? n8p[c][e].y : n8p[c][e].x;
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                xz[c][t >> 1][t & 1] = m ? xzp[c][t >> 1][t & 1].y : xzp[c][t >> 1][t & 1].x;
                                yz[c][t >> 1][t & 1] = m ? yzp[c][t >> 1][t & 1].y : yzp[c][t >> 1][t & 1].x;
                            }
                            mz[c][0] = m ? mzp[c][0].y : mzp[c][0].x;
                            mz[c][1] = m ? mzp[c][1].y : mzp[c][1].x;
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) n8[c][e] = n8_of(m, c, e);
                            const float4 x = tik[m][c], y = tjk[m][c];
                            xz[c][0][0] = x.x; xz[c][0][1] = x.y; xz[c][1][0] = x.z; xz[c][1][1] = x.w;
                            yz[c][0][0] = y.x; yz[c][0][1] = y.y; yz[c][1][0] = y.z; yz[c][1][1] = y.w;
                            mz[c][0] = tmk[m][c].x;
                            mz[c][1] = tmk[m][c].y;
                        }
                    }
                    // most tables lie far above the band: prove it from the table-free
                    // approximation and skip the exact score's log-table gathers
                    if (pruning) {
                        const float bm = kPaired ? (m ? bnd.y : bnd.x)
                                                 : k2_bound_finish(k2_bound_cells<LaneOps1>(n8, rcl, xz, yz, mz));
                        if (__fsub_rn(bm, prune) > fminf(es.tloc, thr_g)) continue;
                    }
                    // a survivor (or every table, without pruning): its exact cells
                    float u0[kCells], u1[kCells];
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        cells_u(n8[c], rcl[c], make_float4(xz[c][0][0], xz[c][0][1], xz[c][1][0], xz[c][1][1]),
                                make_float4(yz[c][0][0], yz[c][0][1], yz[c][1][0], yz[c][1][1]),
                                make_float2(mz[c][0], mz[c][1]), c ? u1 : u0);
                    canon_rows(u0, dsel);
                    canon_rows(u1, dsel);
                    int r0[kCells], r1[kCells];
                    if (!counts_of(u0, u1, pt.n_c[0], pt.n_c[1], r0, r1)) {
                        atomicOr(&ctrl->status, kStBadCount);
                        continue;
                    }
                    const float sc = k2_f32(r0, r1, lf2);
                    if (dbg) dbg[((size_t)i * M + j) * M + k] = sc;
                    if (tsum_on) {
                        sum_h += table_hash(i, j, k, r0, r1);
                        ++sum_n;
                    }
                    if (sc <= fminf(es.tloc, thr_g)) {
                        const int idx = atomicAdd(&es.cnt, 1);
                        if (idx < kCandCap) es.buf[idx] = Cand{sc, i, j, k};
                        else cand_global(cd, Cand{sc, i, j, k});
                    }
                }
            }
            // accumulators read: the four regions go back to the MMA issuer
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < kCmpSets; ++q) mbar_arrive(regE0 + 8 * regs[q]);
            epi_sync<kCmpEpiThreads>();  // every append of this tile is in
            const int cnt = min(es.cnt, kCandCap);
            if (cnt > kPruneAt) {  // uniform: every thread read the same count
                epi_sync<kCmpEpiThreads>();
                const int kept = epi_prune<kCmpEpiThreads>(cd, es, cnt, tid, false);
                if (tid == 0) es.cnt = kept;
            }
        }
        epi_sync<kCmpEpiThreads>();
        epi_prune<kCmpEpiThreads>(cd, es, min(es.cnt, kCandCap), tid, true);
        if (tsum_on) table_sum_flush(cd.tsum, sum_h, sum_n);
    }
    if (prof) {
        if (warp == 0 && lane == 0) atomicAdd(prof + 0, w_acc);
        if (warp == 1 && lane == 0) {
            atomicAdd(prof + 1, w_acc);
            atomicAdd(prof + 2, w_acc2);
            atomicAdd(prof + 7, w_acc3);
        }
        if (threadIdx.x == kCmpEpiWarp0 * 32) {
            atomicAdd(prof + 4, w_acc);
            atomicAdd(prof + 5, (unsigned long long)(clock64() - t_start));
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

}  // namespace

size_t scan_cmp_smem() { return 1024 + kSlots * (kSlotA + kSlotB) + 256 + sizeof(EpiShared) + 64; }

int cmp_tiles_of(int M, int b_lo, int jb_end) {
    const int nb = std::min((M + 63) / 64, jb_end), nk = (M + kTK - 1) / kTK;
    int t = 0;
    for (int jb = b_lo; jb < nb; ++jb) t += nk - 2 * jb;
    return t;
}

cudaError_t launch_compact(const Planes& pl, const CmpFirst* firsts, int i0, int n_first,
                           uint8_t* cmp, cudaStream_t st) {
    if (n_first == 0) return cudaSuccess;
    const dim3 grid((pl.M + 63) / 64, n_first, 2);
    compact_kernel<<<grid, kCompactThreads, 0, st>>>(pl, firsts, i0, cmp);
    return cudaGetLastError();
}

template <bool kInstr, bool kPaired>
static cudaError_t launch_cmp_variant(const CmpArgs& a, int grid, cudaStream_t st) {
    const size_t smem = scan_cmp_smem();
    // once per device: the register split adds up to exactly the launch's registers, so refuse a
    // build whose register count differs (its increase could never be granted); then allow the
    // dynamic shared memory
    static std::atomic<unsigned long long> ready{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(ready.load(std::memory_order_acquire) & bit)) {
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, scan_cmp_kernel<kInstr, kPaired>);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != kCmpRegLaunch) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(scan_cmp_kernel<kInstr, kPaired>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        ready.fetch_or(bit, std::memory_order_release);
    }
    if (a.n_tiles == 0) return cudaSuccess;
    scan_cmp_kernel<kInstr, kPaired><<<grid, kCmpThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// The instrumented instantiation serves table checksums and wait profiles only, so the product
// kernel carries no hook.
cudaError_t launch_scan_cmp(const CmpArgs& a, int grid, cudaStream_t st, bool instrumented, bool paired) {
    if (paired)
        return instrumented ? launch_cmp_variant<true, true>(a, grid, st)
                            : launch_cmp_variant<false, true>(a, grid, st);
    return instrumented ? launch_cmp_variant<true, false>(a, grid, st)
                        : launch_cmp_variant<false, false>(a, grid, st);
}

}  // namespace epi3
