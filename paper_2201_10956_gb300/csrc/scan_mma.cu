// Tensor-core counting scan: the triplet count as a dense contraction on tcgen05.
//
// For a fixed first SNP i and class c the 8 cells with genotypes in {0,1} of every
// triplet (i, j, k) are one GEMM over the class's samples s:
//     D[(j, a, b), (k, z)] = sum_s ([g_i(s) = a] & [g_j(s) = b]) * [g_k(s) = z],
// A = one-hot pair products (4 rows per second SNP), B = one-hot rows of the third SNP
// (2 rows per SNP), both 0/1 values, FP32 accumulation in TMEM (counts < 2^24: exact).
// The other 19 cells follow exactly from pair tables and marginals (derive27), then K2
// and the candidate band exactly as in the POPC scan.  (The paper's kernels use POPCNT,
// Sec. IV; its related work, Sec. II, points at tensor-core formulations.)
//
// Tile = (i, 32 second SNPs, 64 third SNPs): MMA M = 128 rows (j, a, b), N = 128 columns
// (k, z), four tcgen05.mma per step; a step is 256 samples with block-scaled FP4 E2M1
// operands (kind::mxf4, two samples per byte, every scale 2^0), 128 with FP8 E4M3
// (kind::f8f6f4) or 64 with FP16 (kind::f16).  The one-hot matrix is pre-tiled in HBM in the
// exact 128B-swizzled shared-memory image; per step cp.async.bulk fetches the third-SNP chunk
// (the MMA's B operand, read from shared memory), the one-hot rows of the second SNPs (Y) and
// of the first SNP (X).  Four producer warps form A = Y AND X in registers and store it
// straight into tensor memory (tcgen05.st), where the MMA reads it: the product never passes
// through shared memory, whose bandwidth bounded the first design of this kernel.
//
// Tensor memory (512 columns): a ring of three 128-column accumulator regions, one per
// (tile, class) segment, so the epilogue of a tile overlaps the next tile's first class;
// then the A stages (32 columns each: four, or three beside the E2M1 block-scale columns).
// Shared memory: a ring of TMEM stages + 2 steps, the epilogue's candidate buffer and its
// per-warp transpose slabs.
//
// Warp roles: operand loader + TMEM allocator; MMA issuer (one wait and one commit per step);
// 8 epilogue warps (two per TMEM lane quadrant; pair-table rows, TMEM read, transpose, the 19
// derived cells of count + 1 in exact FP32, a table-free bound that skips tables above the
// candidate band, the exact integer table and FP32 K2 for the rest); 4 A producers (one thread
// per TMEM lane; they also return each shared-memory stage to the loader once its MMAs are
// complete).  Two layouts: 14 warps with 128 registers each, or 16 warps whose groups move
// registers to the epilogue (setmaxnreg) for data sets with fewer samples.  Every mbarrier
// wait is bounded; on timeout the kernel records kStTimeout, waits for its own bulk copies,
// frees TMEM and returns.
#include <atomic>

#include "epi3_internal.cuh"
#include "tc_common.cuh"

namespace epi3 {

namespace {

constexpr int kKB = 64;                  // third SNPs per tile (B rows = 2 per SNP)
constexpr int kJB = 32;                  // second SNPs per tile (A rows = 4 per SNP)
// Shared-memory ring of kSmStages slots, one K-step each, every operand's slots contiguous.
// Two consecutive K-steps of one (tile, class) segment that fall on an aligned slot pair (an
// even slot and the next) arrive by ONE bulk copy per operand, signalled on the even slot's
// barrier: every copy costs the SM's copy engine a fixed overhead of about 100 cycles besides
// its bytes, so fewer, larger copies raise the operand intake.  A slot goes back to the loader
// once the MMAs of its K-step are complete.
constexpr int kSmStagesMax = 6;
constexpr int kChunk = 16384;            // bytes of one operand step: 128 rows x 128 B
// Warp roles, two layouts.  Plain form, 14 warps: 0 = operand loader + TMEM allocator, 1 = MMA
// issuer, 2..9 = epilogue (two warps per TMEM lane quadrant), 10..13 = A producers (one thread
// per TMEM lane); every warp has the 128 registers the 14 warps can have.  Register-split
// form, 16 warps in four warp groups: 0 = loader, 1 = MMA issuer (2, 3 idle), 4..7 =
// producers, 8..15 = epilogue; launched with 128 registers per thread (all 65536), after which
// the groups trade them, kRegCtl + kRegProd + 2 kRegEpi = 4 x 128 per thread slot, so that the
// epilogue's working set fits without spills.  The split pays where the epilogue bounds the
// scan (few samples per triplet); with many samples the MMA pipeline bounds it and the plain
// form is faster.
constexpr int kWarpMma = 1;
constexpr int kProdWarps = 4;
constexpr int kEpiWarps = 8, kEpiThreads = kEpiWarps * 32;
template <bool kSplit>
__host__ __device__ constexpr int threads_of() { return kSplit ? 512 : 448; }
template <bool kSplit>
__host__ __device__ constexpr int prod_warp0() { return kSplit ? 4 : 10; }
template <bool kSplit>
__host__ __device__ constexpr int epi_warp0() { return kSplit ? 8 : 2; }
constexpr int kRegLaunch = 128, kRegCtl = 56, kRegProd = 104, kRegEpi = 176;
static_assert(kRegCtl + kRegProd + 2 * kRegEpi == 4 * kRegLaunch, "register split");
static_assert(threads_of<true>() * kRegLaunch == 65536, "the split launch holds the whole register file");
constexpr int kYChunk = kChunk / 2;      // one-hot rows (j, b) of 32 second SNPs: 64 rows
constexpr int kXBytes = 256;             // one-hot rows (i, 0) and (i, 1): 2 rows
constexpr int kTmemCols = 512;
constexpr int kRegions = 3;              // 128-column accumulator regions (columns 0..383)
constexpr uint32_t kProdCol0 = 384;      // A stages: 32 columns (128 bytes of K) each
constexpr uint32_t kProdCols = 32;
constexpr uint32_t kSfCol = 480;         // E2M1 block scales: A at 480..495, B at 496..511
constexpr int kTmStagesMax = 4;
// tensor-memory ring of A stages: four, or three beside the block-scale columns
template <int kKind>
__host__ __device__ constexpr int tm_stages() { return kKind == kKindE2M1 ? 3 : 4; }
template <int kKind>
__host__ __device__ constexpr int sm_stages() { return 6; }
static_assert(kSmStagesMax % 2 == 0, "slot pairs");
static_assert(kRegions * 128 + 4 * kProdCols <= kTmemCols, "tensor memory budget");
static_assert(kRegions * 128 + 3 * kProdCols <= kSfCol, "tensor memory budget (E2M1)");
constexpr int kTRow = 80;                   // bytes per row of an epilogue transpose slab


// D (+)= A * B^T with A (128 rows x 32 bytes of K) in tensor memory at column `a`; the E2M1
// form scales every 32-element block by the UE8M0 factors at `sfa` / `sfb` (all 1.0 here).
template <int kKind>
__device__ __forceinline__ void tc_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc, uint32_t sfa, uint32_t sfb) {
    if (kKind == kKindE4M3) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n"
            ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
    } else if (kKind == kKindF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
            ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3,"
            " [%5], [%6], p;\n}\n"
            ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc), "r"(sfa), "r"(sfb) : "memory");
    }
}
// 32 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
          "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
          "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]),
          "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]),
          "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void epi_bar() {
    asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory");
}
// Barrier of the epilogue threads that also returns whether any of them passed true.
__device__ __forceinline__ bool epi_bar_or(bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, 1, %2, a;\n"
        " selp.u32 %0, 1, 0, b;\n}\n"
        : "=r"(r) : "r"((uint32_t)p), "r"(kEpiThreads) : "memory");
    return r != 0;
}

// Instruction descriptor: FP32 accumulator, A/B E4M3 (kind::f8f6f4) or F16 (kind::f16),
// both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
// Block-scaled form (kind::mxf4): A/B E2M1 (format 1), UE8M0 scales (bit 23), K-major,
// N = 128, M = 128, scale-factor data ids 0.
constexpr uint32_t kIdescMx = (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | (1u << 23) |
                              ((128u >> 4) << 24);
template <int kKind>
__host__ __device__ constexpr uint32_t idesc_of() { return kKind == kKindE2M1 ? kIdescMx : kIdesc; }

// 4 bits -> 4 bytes of value `one` (E4M3 1.0 = 0x38) or 0.
__device__ __forceinline__ uint32_t nib_to_bytes(uint32_t nib, uint32_t one) {
    return ((nib * 0x00204081u) & 0x01010101u) * one;
}
// 2 bits -> 2 FP16 values (1.0 = 0x3C00) packed in one word.
__device__ __forceinline__ uint32_t bits2_to_h2(uint32_t b2) {
    return ((b2 * 0x8001u) & 0x10001u) * 0x3C00u;
}
// One 16-byte operand unit from its sample bits: 32 samples (E2M1), 16 (E4M3) or 8 (FP16).
template <int kKind>
__device__ __forceinline__ uint4 unit_of_bits(uint32_t b) {
    uint4 v;
    if (kKind == kKindE2M1) {
        v.x = byte_to_e2m1(b);
        v.y = byte_to_e2m1(b >> 8);
        v.z = byte_to_e2m1(b >> 16);
        v.w = byte_to_e2m1(b >> 24);
    } else if (kKind == kKindE4M3) {
        v.x = nib_to_bytes(b & 0xF, 0x38u);
        v.y = nib_to_bytes((b >> 4) & 0xF, 0x38u);
        v.z = nib_to_bytes((b >> 8) & 0xF, 0x38u);
        v.w = nib_to_bytes((b >> 12) & 0xF, 0x38u);
    } else {
        v.x = bits2_to_h2(b & 3);
        v.y = bits2_to_h2((b >> 2) & 3);
        v.z = bits2_to_h2((b >> 4) & 3);
        v.w = bits2_to_h2((b >> 6) & 3);
    }
    return v;
}

// Sample bits of one-hot row (c, p, m) for K-step ks, 32 per word in sample order (w[0..7];
// words past the step, the class or the SNPs stay 0, except the class's bias sample).
template <int kKind>
__device__ __forceinline__ void step_words(const Planes& pl, int c, int p, int m, int ks,
                                           uint32_t* w) {
#pragma unroll
    for (int t = 0; t < 8; ++t) w[t] = 0;
    if (m >= pl.M) return;
    const uint4* row = pl.planes + pl.coff[c] + (size_t)p * pl.W4[c] * pl.M + m;
    if (kKind == kKindE2M1) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int w4 = 2 * ks + hh;
            if (w4 < pl.W4[c]) {
                const uint4 g = __ldg(row + (size_t)w4 * pl.M);
                w[4 * hh] = g.x; w[4 * hh + 1] = g.y; w[4 * hh + 2] = g.z; w[4 * hh + 3] = g.w;
            }
        }
    } else if (kKind == kKindE4M3) {
        if (ks < pl.W4[c]) {
            const uint4 g = __ldg(row + (size_t)ks * pl.M);
            w[0] = g.x; w[1] = g.y; w[2] = g.z; w[3] = g.w;
        }
    } else if ((ks >> 1) < pl.W4[c]) {
        const uint4 g = __ldg(row + (size_t)(ks >> 1) * pl.M);
        w[0] = (ks & 1) ? g.z : g.x;
        w[1] = (ks & 1) ? g.w : g.y;
    }
    // the bias sample at class position N_c: a 1 in every row, so every accumulator of the
    // class ends at count + 1 (the K-steps of a class always leave room for it)
    const int sps = kKind == kKindE2M1 ? 256 : (kKind == kKindE4M3 ? 128 : 64);
    const int bias = 128 * pl.W4[c] - pl.pad[c] - ks * sps;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (bias >= 32 * t && bias < 32 * t + 32 && bias < sps) w[t] |= 1u << (bias & 31);
}

// The 128 bytes of one operand row (r of the chunk) in the 128B-swizzled image.
template <int kKind>
__device__ __forceinline__ void store_row(uint8_t* tile, uint32_t r, const uint32_t* w) {
#pragma unroll
    for (uint32_t u = 0; u < 8; ++u) {
        uint32_t b;
        if (kKind == kKindE2M1) b = w[u];
        else if (kKind == kKindE4M3) b = (w[u >> 1] >> ((u & 1) * 16)) & 0xFFFFu;
        else b = (w[u >> 2] >> ((u & 3) * 8)) & 0xFFu;
        *reinterpret_cast<uint4*>(tile + sw128_off(r, u)) = unit_of_bits<kKind>(b);
    }
}

// Walks one CTA's sequence of (tile, class, K-step): tiles blockIdx.x + n * gridDim.x,
// class 0 then class 1, K-steps of the tile's cohort (classes without samples skipped).
struct StepCursor {
    long long tl;
    int c, ks, ks0, ks1;
    int4 tile;
    const CohortDev* cd;
    bool valid;
};

__device__ __forceinline__ void cursor_load(StepCursor& cu, const CohortDev* cds, const int4* tiles,
                                            long long my_tiles) {
    cu.valid = cu.tl < my_tiles;
    if (!cu.valid) return;
    cu.tile = tiles[blockIdx.x + cu.tl * gridDim.x];
    cu.cd = cds + cu.tile.w;
    cu.ks0 = cu.cd->KS[0];
    cu.ks1 = cu.cd->KS[1];
    cu.c = cu.ks0 > 0 ? 0 : 1;
    cu.ks = 0;
}

// Advance by n K-steps (the steps of one shared-memory stage, never past its segment).
__device__ __forceinline__ void cursor_next(StepCursor& cu, const CohortDev* cds, const int4* tiles,
                                            long long my_tiles, int n) {
    if (!cu.valid) return;
    cu.ks += n;
    if (cu.ks < (cu.c ? cu.ks1 : cu.ks0)) return;
    if (cu.c == 0 && cu.ks1 > 0) {
        cu.c = 1;
        cu.ks = 0;
        return;
    }
    ++cu.tl;
    cursor_load(cu, cds, tiles, my_tiles);
}

template <int kKind, bool kProf, bool kSplit>
__global__ void __launch_bounds__(threads_of<kSplit>(), 1)
scan_mma_kernel(const CohortDev* __restrict__ cds, const int4* __restrict__ tiles, long long n_tiles,
                unsigned long long* __restrict__ prof) {
    // prof (optional): per role, cycles spent waiting, summed over CTAs:
    //   [0] loader on empty stages, [1] MMA on full stages, [2] MMA on free accumulator
    //   regions, [3] producers (lane 0 of each producer warp) on full stages, [4] epilogue
    //   (lane 0 of each epilogue warp) on full accumulators, [5] kernel cycles of this CTA,
    //   [6] producers on free tensor-memory stages, [7] MMA issuer issuing MMAs and commits
    const long long t_start = kProf ? clock64() : 0;
    unsigned long long w_acc = 0, busy = 0, w_acc2 = 0;
    unsigned long long* my_acc = kProf ? &w_acc : nullptr;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned stage buffers (the 128B swizzle pattern is anchored there)
    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr int kTm = tm_stages<kKind>();
    constexpr int kSmStages = sm_stages<kKind>();
    uint8_t* sK = base;                                    // [kSmStages][16 KB] third-SNP rows
    uint8_t* sY = base + kSmStages * kChunk;               // [kSmStages][8 KB]
    uint8_t* sX = sY + kSmStages * kYChunk;                // [kSmStages][256 B]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sX + kSmStages * kXBytes);
    // bars: fullS[kSmStages], emptyS[kSmStages] (shared-memory ring), fullT[4], emptyT[4]
    // (tensor-memory A ring), acc_full[2], reg_free[3], drain
    constexpr int kNBars = 2 * kSmStages + 2 * kTmStagesMax + 6;
    static_assert(kNBars * 8 + 8 <= 256, "barrier area");
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kNBars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    EpiShared& es = *reinterpret_cast<EpiShared*>(reinterpret_cast<uint8_t*>(bars) + 256);
    uint8_t* sT = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(&es) + sizeof(EpiShared) + 15) & ~static_cast<uintptr_t>(15));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kProdWarp0 = prod_warp0<kSplit>(), kEpiWarp0 = epi_warp0<kSplit>();
    const bool is_ctl = kSplit ? warp < kProdWarp0 : warp < kEpiWarp0;
    const bool is_prod = warp >= kProdWarp0 && warp < kProdWarp0 + kProdWarps;
    const uint32_t fullS0 = smem_u32(bars), emptyS0 = smem_u32(bars + kSmStages),
                   fullT0 = smem_u32(bars + 2 * kSmStages),
                   emptyT0 = smem_u32(bars + 2 * kSmStages + kTmStagesMax),
                   accF0 = smem_u32(bars + 2 * kSmStages + 2 * kTmStagesMax),
                   regE0 = accF0 + 16, drain0 = accF0 + 40;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSmStages; ++s) {
            mbar_init(fullS0 + 8 * s, 1);
            mbar_init(emptyS0 + 8 * s, 1);
        }
        for (int s = 0; s < kTmStagesMax; ++s) {
            mbar_init(fullT0 + 8 * s, kProdWarps);  // one arrival per producer warp
            mbar_init(emptyT0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) mbar_init(accF0 + 8 * b, 1);
        for (int r = 0; r < kRegions; ++r) mbar_init(regE0 + 8 * r, kEpiWarps);
        mbar_init(drain0, 1);
        *abort_flag = 0;
        es.cnt = 0;
        es.tloc = __int_as_float(0x7f800000);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long my_tiles =
        n_tiles > blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto fail = [&](const CohortDev* cd) {
        *abort_flag = 1;
        atomicOr(&cd->ctrl->status, kStTimeout);
    };

    if (is_ctl) {
        if (kSplit) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegCtl));
        if (warp == 0) {
            // ------------------------------------------------ operand loader (lane 0)
            if (lane == 0) {
                StepCursor cu{};
                cu.tl = 0;
                cursor_load(cu, cds, tiles, my_tiles);
                Ring rs{0, 0u};
                uint32_t used = 0, fph = 0;  // slots whose full barrier was used / their parity
                while (cu.valid) {
                    const int s = rs.s;
                    const int nks = cu.c ? cu.ks1 : cu.ks0;
                    // an even slot and the next take two steps of one segment in one copy
                    const int n = ((s & 1) == 0 && cu.ks + 1 < nks) ? 2 : 1;
                    if (!mbar_wait_t(emptyS0 + 8 * s, rs.ph ^ 1u, abort_flag, my_acc) ||
                        (n == 2 && !mbar_wait_t(emptyS0 + 8 * (s + 1), rs.ph ^ 1u, abort_flag, my_acc))) {
                        fail(cu.cd);
                        break;
                    }
                    // K: one-hot rows (k, z) of the tile's 64 third SNPs; Y: rows (j, b) of its 32
                    // second SNPs; X: rows (i, 0), (i, 1).  Each for the n consecutive K-steps,
                    // contiguous in its array, so one bulk copy apiece.
                    const long long ca = (cu.c ? cu.cd->oh_off1 : 0) + (long long)cu.tile.z * nks + cu.ks;
                    const long long cy = (cu.c ? cu.cd->yoh_off1 : 0) + (long long)cu.tile.y * nks + cu.ks;
                    const long long cx = (cu.c ? cu.cd->xoh_off1 : 0) + (long long)cu.tile.x * nks + cu.ks;
                    const uint32_t fb = fullS0 + 8 * s;
                    mbar_arrive_tx(fb, (unsigned)(n * (kChunk + kYChunk + kXBytes)));
                    bulk_g2s(smem_u32(sK + s * kChunk), cu.cd->oh + ca * kChunk, (unsigned)(n * kChunk), fb);
                    bulk_g2s(smem_u32(sY + s * kYChunk), cu.cd->yoh + cy * kYChunk, (unsigned)(n * kYChunk), fb);
                    bulk_g2s(smem_u32(sX + s * kXBytes), cu.cd->xoh + cx * kXBytes, (unsigned)(n * kXBytes), fb);
                    used |= 1u << s;
                    fph ^= 1u << s;
                    ring_next(rs, kSmStages);
                    if (n == 2) ring_next(rs, kSmStages);
                    cursor_next(cu, cds, tiles, my_tiles, n);
                }
                // drain: the copies issued must land before the CTA exits (each used barrier's
                // last phase)
                for (int b = 0; b < kSmStages; ++b) {
                    if (!((used >> b) & 1u)) continue;
                    volatile int no_abort = 0;
                    mbar_wait(fullS0 + 8 * b, ((fph >> b) & 1u) ^ 1u, &no_abort);
                }
            }
        } else if (warp == kWarpMma) {
            // ------------------------------------------------ MMA issuer (lane 0)
            if (lane == 0) {
                bool ok = true;
                if (cds[0].inject_timeout) {  // test hook: a wait that can only run out (about 1 s)
                    if (!mbar_wait(drain0, 0, abort_flag)) fail(cds);
                    ok = false;
                }
                // The issuing thread's own instruction latency bounds the step rate, so the loop
                // keeps its stage addresses and phases as incrementally updated registers.
                Ring rR{0, 0u};
                const uint64_t db0 = sw128_desc(smem_u32(sK));
                uint64_t db = db0;                        // B descriptor of shared-memory stage s
                int s = 0, t = 0;                         // shared-memory / TMEM stage
                uint32_t phT = 0, fT = fullT0, eT = emptyT0, ta = tmem + kProdCol0;
                for (long long tl = 0; tl < my_tiles && ok; ++tl) {
                    const int4 tile = tiles[blockIdx.x + tl * gridDim.x];
                    const CohortDev* cd = cds + tile.w;
                    const int KS[2] = {cd->KS[0], cd->KS[1]};
                    for (int c = 0; c < 2 && ok; ++c) {
                        // accumulator region of segment (tile, class): a ring of kRegions
                        if (!mbar_wait_t(regE0 + 8 * rR.s, rR.ph ^ 1u, abort_flag, kProf ? &busy : nullptr)) {
                            fail(cd);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)rR.s * 128u;
                        ring_next(rR, kRegions);
                        for (int ks = 0; ks < KS[c]; ++ks) {
                            // the producers arrive on fullT only after they saw the step's bulk
                            // copies land (fullS), so one wait covers both operands
                            if (!mbar_wait_t(fT, phT, abort_flag, my_acc)) {
                                fail(cd);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const long long t_issue = kProf ? clock64() : 0;
                            tc_mma_ts<kKind>(d, ta, db, idesc_of<kKind>(), ks > 0 ? 1u : 0u,
                                             tmem + kSfCol, tmem + kSfCol + 16);
    #pragma unroll
                            for (int kk = 1; kk < 4; ++kk)  // 32 bytes of K per instruction
                                tc_mma_ts<kKind>(d, ta + 8 * kk, db + 2 * kk, idesc_of<kKind>(), 1u,
                                                 tmem + kSfCol, tmem + kSfCol + 16);
                            // one commit per step: its arrival frees the TMEM A stage, and the
                            // producers then release the shared-memory stage to the loader
                            tc_commit(eT);
                            if (kProf) w_acc2 += (unsigned long long)(clock64() - t_issue);
                            if (++t == kTm) {
                                t = 0;
                                phT ^= 1u;
                                fT = fullT0;
                                eT = emptyT0;
                                ta = tmem + kProdCol0;
                            } else {
                                fT += 8;
                                eT += 8;
                                ta += kProdCols;
                            }
                            if (++s == kSmStages) {
                                s = 0;
                                db = db0;
                            } else {
                                db += (uint64_t)(kChunk >> 4);
                            }
                        }
                    }
                    if (ok) tc_commit(accF0 + 8 * (int)(tl & 1));
                }
                // every MMA issued must complete before TMEM is released
                tc_commit(drain0);
                volatile int no_abort = 0;
                mbar_wait(drain0, 0, &no_abort);
            }
    }
    } else if (is_prod) {
        if (kSplit) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegProd));
        // ------------------------------------------------ producers: TMEM lane L = (jj, a, b)
        // Product row (j, a, b) = one-hot row (j, b) AND one-hot row (i, a), bit by bit (an
        // element is 1.0 or 0 in every kind, and 1.0 AND 1.0 = 1.0), read from the staged Y and
        // X rows (swizzled) and stored in natural K order into this step's TMEM columns, where
        // the MMA reads it as its A operand.
        const int L = 32 * (warp & 3) + lane;
        const int jj = L >> 2, ga = (L >> 1) & 1, gb = L & 1;
        const uint32_t yr = (uint32_t)(2 * jj + gb);
        const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
        const uint32_t tl_base = tmem + lane_off + kProdCol0;
        if (kKind == kKindE2M1) {
            // block scale factors 2^0 (UE8M0 127) in every byte of the scale columns; ordered
            // before the first MMA by this warp's first fullT arrival
            uint32_t one[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) one[t] = 0x7F7F7F7Fu;
            tc_st32(tmem + lane_off + kSfCol, one);
            tc_wait_st();
        }
        // Software pipeline: step q's shared-memory loads are issued before the wait for step
        // q-1's tensor-memory store, so the two latencies overlap.  Plain tile and step
        // loops with ring counters keep the per-step bookkeeping to a few integer operations.
        int t_prev = -1;  // TMEM stage of a store issued but not yet published
        Ring rS{0, 0u}, rT{0, 0u};
        Ring rF{0, 0u};   // shared-memory slot of step q - kTm (released once its MMAs finish)
        int warm = 0;     // min(q, kTm)
        uint32_t fph = 0; // parity of each slot's full barrier (toggled when a copy's last step is read)
        bool ok = true;
        for (long long tl = 0; tl < my_tiles && ok; ++tl) {
            const int4 tile = tiles[blockIdx.x + tl * gridDim.x];
            const CohortDev* cd = cds + tile.w;
            const int KS0 = cd->KS[0], KS1 = cd->KS[1];
            const int nsteps = KS0 + KS1;
            const uint32_t xp = (2u * (uint32_t)(tile.x & 63) + (uint32_t)ga) & 7u;
            const uint8_t* xrow = sX + ga * 128;
            for (int q = 0; q < nsteps; ++q) {
                const int s = rS.s, t = rT.s;
                // the loader's pairing rule: an odd slot whose step follows one of the same segment
                // arrived with it, on the even slot's barrier; a step on an even slot whose next
                // step is in the same segment shares its copy with that step
                const bool second = (s & 1) && q > 0 && q != KS0;
                const bool first_of_two = !(s & 1) && q + 1 < nsteps && q + 1 != KS0;
                const int fb = second ? s - 1 : s;
                // the MMAs of step q - kTm have read TMEM stage t; the loader's copy of step q
                // has landed
                const bool got =
                    mbar_wait_t(emptyT0 + 8 * t, rT.ph ^ 1u, abort_flag, kProf ? &w_acc2 : nullptr) &&
                    mbar_wait_t(fullS0 + 8 * fb, (fph >> fb) & 1u, abort_flag, my_acc);
                if (!first_of_two) fph ^= 1u << fb;
                // tcgen05.st is warp-collective: the whole warp goes on or stops together
                if (!__all_sync(0xffffffffu, got)) {
                    fail(cd);
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (warm == kTm) {  // step q - kTm is complete: its slot goes back to the loader
                    if (warp == kProdWarp0 && lane == 0) mbar_arrive(emptyS0 + 8 * rF.s);
                    ring_next(rF, kSmStages);
                } else {
                    ++warm;
                }
                const uint8_t* ys = sY + s * kYChunk;
                const uint8_t* xs = xrow + s * kXBytes;
                uint4 y[8], x[8];
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u) {
                    y[u] = *reinterpret_cast<const uint4*>(ys + sw128_off(yr, u));
                    x[u] = *reinterpret_cast<const uint4*>(xs + ((u ^ xp) << 4));
                }
                if (t_prev >= 0) {  // publish step q-1: every lane's store is done, one arrival
                    tc_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(fullT0 + 8 * t_prev);
                }
                uint32_t v[32];
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u) {
                    v[4 * u + 0] = y[u].x & x[u].x;
                    v[4 * u + 1] = y[u].y & x[u].y;
                    v[4 * u + 2] = y[u].z & x[u].z;
                    v[4 * u + 3] = y[u].w & x[u].w;
                }
                tc_st32(tl_base + (uint32_t)t * kProdCols, v);
                t_prev = t;
                ring_next(rS, kSmStages);
                ring_next(rT, kTm);
            }
        }
        if (t_prev >= 0) {  // the last store (also on the abort path: nothing left in flight)
            tc_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(fullT0 + 8 * t_prev);
        }
    } else {
        if (kSplit) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegEpi));
        // ------------------------------------------------ epilogue
        // TMEM lane L = (jj, a, b) holds, per class, the counts of (i = a, j = b, k = z) for
        // every column 2 kk + z.  The four lanes of one jj exchange values so that each ends
        // with all 8 cells of two (jj, kk) per 16-column group.
        const int tid = threadIdx.x - kEpiWarp0 * 32;   // 0..255
        const int quad = warp & 3, half = (warp - kEpiWarp0) >> 2;  // TMEM lane quadrant
        const int jj = 8 * quad + (lane >> 2), me = lane & 3;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint8_t* tw = sT + (warp - kEpiWarp0) * (32 * kTRow);  // this warp's transpose slab
        int cur = -1;
        unsigned long long sum_h = 0, sum_n = 0;  // table checksum of this thread (tsum_on)
        Ring rR{0, 0u};
        for (long long tl = 0; tl < my_tiles; ++tl) {
            const int buf = (int)(tl & 1);
            const int4 tile = tiles[blockIdx.x + tl * gridDim.x];
            const CohortDev& cd = cds[tile.w];
            if (tile.w != cur) {  // candidates are per cohort: flush the previous one's
                epi_bar();  // the previous tile's count is settled
                if (cur >= 0) epi_prune<kEpiThreads>(cds[cur], es, min(es.cnt, kCandCap), tid, true);
                if (tid == 0) {
                    es.cnt = 0;
                    es.tloc = __int_as_float(0x7f800000);
                }
                cur = tile.w;
            }
            const int M = cd.pl.M;
            const int i = tile.x, j = tile.y * kJB + jj, kb0 = tile.z * kKB;
            // plain form: one thread polls the accumulators' barrier and the other epilogue
            // warps wait at the named barrier below, which costs no shared-memory traffic
            // (there the epilogue waits for the MMA pipeline, and polling from all eight warps
            // competes with the producers' shared-memory reads); the split form's epilogue
            // bounds the scan, and every warp polls so that none waits for a wake-up
            bool bad = false;
            if (kSplit || tid == 0) {
                bad = !mbar_wait_t(accF0 + 8 * buf, (unsigned)((tl >> 1) & 1), abort_flag, my_acc);
                if (bad) fail(&cd);
            }
            // uniform decision (every epilogue thread stops on the same tile); also orders the
            // previous tile's candidate bookkeeping before this tile's appends, and the
            // barrier's completion, observed by thread 0, before every thread's TMEM reads
            if (epi_bar_or(bad || *abort_flag)) break;
            tc_fence_after();
            const int KS0 = cd.KS[0], KS1 = cd.KS[1];
            const PairTables pt = cd.pt;
            long long pij = -1;
            if (j < M && j > i) {
                pij = pair_index(i, j);
                if (pij < cd.pair_begin || pij >= cd.pair_end) pij = -1;
            }
            const bool jrow = pij >= 0;
            int4 pxy[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
            int2 my[2] = {make_int2(0, 0), make_int2(0, 0)}, mx[2];
            if (jrow) {
                pxy[0] = __ldg(pt.pt + pij);
                pxy[1] = __ldg(pt.pt + pt.n_pairs + pij);
                my[0] = __ldg(pt.marg + j);
                my[1] = __ldg(pt.marg + M + j);
            }
            mx[0] = __ldg(pt.marg + i);
            mx[1] = __ldg(pt.marg + M + i);
            const RowCells rcl[2] = {row_cells(pxy[0], mx[0], my[0], pt.n_c[0]),
                                     row_cells(pxy[1], mx[1], my[1], pt.n_c[1])};
            const int reg0 = rR.s;
            ring_next(rR, kRegions);
            const int reg1 = rR.s;
            ring_next(rR, kRegions);
            const uint32_t rc[2] = {(uint32_t)reg0 * 128u, (uint32_t)reg1 * 128u};
            const float2* lf2 = cd.k2.lf2;
            const float prune = cd.k2.prune_delta;
            float* dbg = cd.dbg;
            Ctrl* ctrl = cd.ctrl;
            for (int gi = 0; gi < 4; ++gi) {
                const int g = half + 2 * gi;            // 16-column group = 8 third SNPs
                // the global band threshold only shrinks: a copy read once per group is a
                // valid (looser) filter
                const float thr_g = __uint_as_float(*(volatile unsigned*)&ctrl->thr);
                // this lane's two triplets (k = kb0 + 8 g + 2 me + m): their pair-table rows
                // are requested first, so the loads overlap the TMEM read and the transpose
                // (an index outside the triangle reads entry 0 and is not used)
                float4 tik[2][2], tjk[2][2];
                float2 tmk[2][2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = kb0 + 8 * g + 2 * me + m;
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
                uint32_t v[2][16];
#pragma unroll
                for (int c = 0; c < 2; ++c) tc_ld16(tmem + lane_base + rc[c] + 16 * g, v[c]);
                tc_wait_ld();
                // n8[c][m][4a + 2b + z] = count + 1 for this lane's third SNPs kk = 8 g + 2 me + m
                // (the accumulators include the bias sample; a class without samples has no
                // K-steps and reads as 1)
                float n8[2][2][8];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const bool has = c ? KS1 > 0 : KS0 > 0;
                    uint32_t x[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) x[t] = has ? v[c][t] : 0x3F800000u;
                    // x[4 blk + e]: column 16 g + 4 blk + e; lane `me` needs block `me` of all
                    // four lanes of its jj.  Through this warp's shared-memory slab: row = lane,
                    // 16-byte unit = block (rows 80 bytes apart, so neither the stores nor the
                    // loads below conflict); row 4 jjl + src then holds cells (a, b) = src.
                    __syncwarp();  // the previous class's loads are done
#pragma unroll
                    for (int blk = 0; blk < 4; ++blk)
                        *reinterpret_cast<uint4*>(tw + lane * kTRow + blk * 16) =
                            make_uint4(x[4 * blk], x[4 * blk + 1], x[4 * blk + 2], x[4 * blk + 3]);
                    __syncwarp();
#pragma unroll
                    for (int src = 0; src < 4; ++src) {
                        const float4 q = *reinterpret_cast<const float4*>(
                            tw + (4 * (lane >> 2) + src) * kTRow + me * 16);
                        n8[c][0][2 * src] = q.x;      // (m = 0, z = 0)
                        n8[c][0][2 * src + 1] = q.y;  // (m = 0, z = 1)
                        n8[c][1][2 * src] = q.z;      // (m = 1, z = 0)
                        n8[c][1][2 * src + 1] = q.w;  // (m = 1, z = 1)
                    }
                }
                // the instrumented instantiation (kProf) also serves table checksums
                const bool tsum_on = kProf && cd.tsum != nullptr;
                const bool pruning = !dbg && !tsum_on && prune > 0.f;
                // the split form has the registers to bound both tables of the lane at once
                // (a lane outside the triangle computes a bound it does not use)
                float bnd[2] = {0.f, 0.f};
                if (kSplit && pruning) {
                    float u0a[kCells], u1a[kCells], u0b[kCells], u1b[kCells];
                    cells_u(n8[0][0], rcl[0], tik[0][0], tjk[0][0], tmk[0][0], u0a);
                    cells_u(n8[1][0], rcl[1], tik[0][1], tjk[0][1], tmk[0][1], u1a);
                    cells_u(n8[0][1], rcl[0], tik[1][0], tjk[1][0], tmk[1][0], u0b);
                    cells_u(n8[1][1], rcl[1], tik[1][1], tjk[1][1], tmk[1][1], u1b);
                    k2_bound_u2(u0a, u1a, u0b, u1b, bnd);
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int k = kb0 + 8 * g + 2 * me + m;
                    if (!(jrow && k > j && k < M)) continue;
                    if (kSplit && pruning && __fsub_rn(bnd[m], prune) > fminf(es.tloc, thr_g))
                        continue;
                    float u0[kCells], u1[kCells];
                    cells_u(n8[0][m], rcl[0], tik[m][0], tjk[m][0], tmk[m][0], u0);
                    cells_u(n8[1][m], rcl[1], tik[m][1], tjk[m][1], tmk[m][1], u1);
                    // most tables lie far above the band: prove it from the table-free
                    // approximation and skip the exact score's 81 log-table gathers
                    if (!kSplit && pruning &&
                        __fsub_rn(k2_bound_u(u0, u1), prune) > fminf(es.tloc, thr_g))
                        continue;
                    // exact integer table; a cell outside [0, N_c] would mean a corrupt count
                    // and is reported instead of looked up
                    int r0[kCells], r1[kCells];
                    if (!counts_of(u0, u1, pt.n_c[0], pt.n_c[1], r0, r1)) {
                        atomicOr(&ctrl->status, kStBadCount);
                        continue;
                    }
                    const float s = k2_f32(r0, r1, lf2);
                    if (dbg) dbg[((size_t)i * M + j) * M + k] = s;
                    if (tsum_on) {
                        sum_h += table_hash(i, j, k, r0, r1);
                        ++sum_n;
                    }
                    if (s <= fminf(es.tloc, thr_g)) {
                        const int idx = atomicAdd(&es.cnt, 1);
                        if (idx < kCandCap) es.buf[idx] = Cand{s, i, j, k};
                        else cand_global(cd, Cand{s, i, j, k});
                    }
                }
            }
            // accumulators read: release both regions to the MMA issuer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(regE0 + 8 * reg0);
                mbar_arrive(regE0 + 8 * reg1);
            }
            epi_bar();  // every append of this tile is in
            const int cnt = min(es.cnt, kCandCap);
            if (cnt > kPruneAt) {  // uniform: every thread read the same count
                epi_bar();
                const int kept = epi_prune<kEpiThreads>(cd, es, cnt, tid, false);
                if (tid == 0) es.cnt = kept;
            }
        }
        epi_bar();
        if (cur >= 0) epi_prune<kEpiThreads>(cds[cur], es, min(es.cnt, kCandCap), tid, true);
        if (kProf && cur >= 0 && cds[cur].tsum) table_sum_flush(cds[cur].tsum, sum_h, sum_n);
    }
    if (kProf && prof) {
        const unsigned long long total = (unsigned long long)(clock64() - t_start);
        if (warp == 0 && lane == 0) atomicAdd(prof + 0, w_acc);
        if (warp == kWarpMma && lane == 0) {
            atomicAdd(prof + 1, w_acc);
            atomicAdd(prof + 2, busy);
            atomicAdd(prof + 7, w_acc2);
        }
        if (is_prod && lane == 0) {
            atomicAdd(prof + 3, w_acc);
            atomicAdd(prof + 6, w_acc2);
        }
        if (!is_ctl && !is_prod && lane == 0) atomicAdd(prof + 4, w_acc);
        if (threadIdx.x == 0) atomicAdd(prof + 5, total);
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols) : "memory");
    }
}

// Pre-tiled one-hot chunks: chunk (c, kb, ks) holds rows r = 2 kk + z (third SNP
// 64 kb + kk, genotype z) over the K-step's samples, already in the swizzled image.
template <int kKind>
__global__ void onehot_kernel(Planes pl, uint8_t* __restrict__ oh, long long off1, int KS0, int KS1,
                              int kb_count) {
    const long long total = ((long long)kb_count * (KS0 + KS1)) * 128;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t & 127);
        const long long ch = t >> 7;  // chunk, in (class, kb, ks) order
        int c, kb, ks;
        if (ch < (long long)kb_count * KS0) {
            c = 0;
            kb = (int)(ch / KS0);
            ks = (int)(ch % KS0);
        } else {
            const long long q = ch - (long long)kb_count * KS0;
            c = 1;
            kb = (int)(q / KS1);
            ks = (int)(q % KS1);
        }
        const int m = kb * kKB + (r >> 1), p = r & 1;
        uint32_t w[8];
        step_words<kKind>(pl, c, p, m, ks, w);
        uint8_t* tile = oh + (c ? off1 + (long long)kb * KS1 + ks : (long long)kb * KS0 + ks) * kChunk;
        store_row<kKind>(tile, (uint32_t)r, w);
    }
}

// Two rearranged copies of the one-hot chunks, so that every operand of a shared-memory stage
// (kStageKs consecutive K-steps) is one contiguous bulk copy:
//   yoh: the rows (j, b) of 32 second SNPs, [class][32-SNP block][K-step], 8 KB each (the half
//        of the 64-SNP chunk that holds them);
//   xoh: the two rows (i, 0), (i, 1) of one first SNP, [class][SNP][K-step], 256 B each (as
//        they sit in the swizzled chunk: an aligned pair of rows of one 8-row group).
__global__ void onehot_views_kernel(const uint8_t* __restrict__ oh, long long off1, int KS0, int KS1,
                                    int kb_count, int M, uint8_t* __restrict__ yoh,
                                    uint8_t* __restrict__ xoh) {
    const long long nks = KS0 + KS1;
    const long long ny = (long long)2 * kb_count * nks * (kYChunk / 16);   // uint4 units of yoh
    const long long nx = (long long)M * nks * (kXBytes / 16);             // uint4 units of xoh
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ny + nx;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < ny) {
            const long long piece = t / (kYChunk / 16), u = t % (kYChunk / 16);
            // piece in [class][jb32][ks] order
            const int c = piece < 2LL * kb_count * KS0 ? 0 : 1;
            const long long p = c ? piece - 2LL * kb_count * KS0 : piece;
            const int KS = c ? KS1 : KS0;
            const long long jb32 = p / KS, ks = p % KS;
            const long long chunk = (c ? off1 + (jb32 >> 1) * KS1 : (jb32 >> 1) * KS0) + ks;
            reinterpret_cast<uint4*>(yoh)[t] = reinterpret_cast<const uint4*>(
                oh + chunk * kChunk + (jb32 & 1) * kYChunk)[u];
        } else {
            const long long tx = t - ny;
            const long long piece = tx / (kXBytes / 16), u = tx % (kXBytes / 16);
            // piece in [class][i][ks] order
            const int c = piece < (long long)M * KS0 ? 0 : 1;
            const long long p = c ? piece - (long long)M * KS0 : piece;
            const int KS = c ? KS1 : KS0;
            const long long i = p / KS, ks = p % KS;
            const long long chunk = (c ? off1 + (i >> 6) * KS1 : (i >> 6) * KS0) + ks;
            const uint32_t xr = 2u * (uint32_t)(i & 63);
            reinterpret_cast<uint4*>(xoh)[tx] = reinterpret_cast<const uint4*>(
                oh + chunk * kChunk + (xr >> 3) * 1024 + (xr & 7) * 128)[u];
        }
    }
}

// Tile list of a whole scan on the device: block b = {kb, jb, count, offset} of (third-SNP
// block, second-SNP block) gets tiles (i, jb, kb, cohort) for i = 0 .. count-1 at offset + i.
__global__ void tile_list_kernel(const int4* __restrict__ blocks, int cohort, int4* __restrict__ tiles) {
    const int4 b = blocks[blockIdx.x];
    for (int i = threadIdx.x; i < b.z; i += blockDim.x) tiles[b.w + i] = make_int4(i, b.y, b.x, cohort);
}

}  // namespace

size_t scan_mma_smem(int kind) {
    const int sm = kind == kKindE2M1 ? sm_stages<kKindE2M1>() : sm_stages<kKindE4M3>();
    return 1024 + sm * (kChunk + kYChunk + kXBytes) + 256 + sizeof(EpiShared) + 16 +
           kEpiWarps * 32 * kTRow + 64;
}

int mma_samples_per_step(int kind) {
    return kind == kKindE2M1 ? 256 : (kind == kKindE4M3 ? 128 : 64);
}

cudaError_t launch_tile_list(const int4* blocks, int n_blocks, int cohort, int4* tiles,
                             cudaStream_t st) {
    if (n_blocks == 0) return cudaSuccess;
    tile_list_kernel<<<n_blocks, 256, 0, st>>>(blocks, cohort, tiles);
    return cudaGetLastError();
}

size_t onehot_bytes(int M, int KS0, int KS1) {
    const size_t kbc = (size_t)(M + 63) / 64, nks = (size_t)KS0 + KS1;
    return kbc * nks * kChunk + 2 * kbc * nks * kYChunk + (size_t)M * nks * kXBytes;
}

cudaError_t launch_onehot_views(const uint8_t* oh, long long off1, int KS0, int KS1, int kb_count,
                                int M, uint8_t* yoh, uint8_t* xoh, cudaStream_t st) {
    const long long units = ((long long)2 * kb_count * (KS0 + KS1) * (kYChunk / 16)) +
                            ((long long)M * (KS0 + KS1) * (kXBytes / 16));
    if (units == 0) return cudaSuccess;
    const long long want = (units + 255) / 256;
    const int blocks = (int)(want < 65535LL * 8 ? want : 65535LL * 8);
    onehot_views_kernel<<<blocks, 256, 0, st>>>(oh, off1, KS0, KS1, kb_count, M, yoh, xoh);
    return cudaGetLastError();
}

cudaError_t launch_onehot(const Planes& pl, uint8_t* oh, long long off1, int KS0, int KS1,
                          int kb_count, int kind, cudaStream_t st) {
    const long long total = ((long long)kb_count * (KS0 + KS1)) * 128;
    const int blocks = (int)((total + 255) / 256 < 65535 * 8 ? (total + 255) / 256 : 65535 * 8);
    if (total == 0) return cudaSuccess;
    if (kind == kKindE2M1)
        onehot_kernel<kKindE2M1><<<blocks, 256, 0, st>>>(pl, oh, off1, KS0, KS1, kb_count);
    else if (kind == kKindE4M3)
        onehot_kernel<kKindE4M3><<<blocks, 256, 0, st>>>(pl, oh, off1, KS0, KS1, kb_count);
    else
        onehot_kernel<kKindF16><<<blocks, 256, 0, st>>>(pl, oh, off1, KS0, KS1, kb_count);
    return cudaGetLastError();
}

template <int kKind, bool kProf, bool kSplit>
static cudaError_t launch_variant(const CohortDev* cohorts, const int4* tiles, long long n_tiles,
                                  int grid, cudaStream_t st, unsigned long long* prof) {
    const size_t smem = scan_mma_smem(kKind);
    // once per device: the warp groups' register split adds up to exactly the launch's
    // registers, so refuse a build whose register count differs (its increase could never be
    // granted); then allow the dynamic shared memory
    static std::atomic<unsigned long long> ready{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(ready.load(std::memory_order_acquire) & bit)) {
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, scan_mma_kernel<kKind, kProf, kSplit>);
        if (e != cudaSuccess) return e;
        if (kSplit && fa.numRegs != kRegLaunch) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(scan_mma_kernel<kKind, kProf, kSplit>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ready.fetch_or(bit, std::memory_order_release);
    }
    scan_mma_kernel<kKind, kProf, kSplit><<<grid, threads_of<kSplit>(), smem, st>>>(cohorts, tiles,
                                                                                 n_tiles, prof);
    return cudaGetLastError();
}

// Role profiling (option "profile") and table checksums use a separate, instrumented
// instantiation, so the normal kernel's hot loops carry no clock reads or hooks.
template <int kKind>
static cudaError_t launch_kind(const CohortDev* cohorts, const int4* tiles, long long n_tiles,
                               int grid, cudaStream_t st, unsigned long long* prof, bool split,
                               bool instrument) {
    if (split)
        return instrument ? launch_variant<kKind, true, true>(cohorts, tiles, n_tiles, grid, st, prof)
                          : launch_variant<kKind, false, true>(cohorts, tiles, n_tiles, grid, st, prof);
    return instrument ? launch_variant<kKind, true, false>(cohorts, tiles, n_tiles, grid, st, prof)
                      : launch_variant<kKind, false, false>(cohorts, tiles, n_tiles, grid, st, prof);
}


int mma_threads(bool split) { return split ? threads_of<true>() : threads_of<false>(); }

cudaError_t launch_scan_mma(const CohortDev* cohorts, const int4* tiles, long long n_tiles,
                            int kind, int grid, cudaStream_t st, unsigned long long* prof,
                            bool split, bool checksum) {
    const bool ins = prof != nullptr || checksum;
    if (kind == kKindE2M1)
        return launch_kind<kKindE2M1>(cohorts, tiles, n_tiles, grid, st, prof, split, ins);
    if (kind == kKindE4M3)
        return launch_kind<kKindE4M3>(cohorts, tiles, n_tiles, grid, st, prof, split, ins);
    return launch_kind<kKindF16>(cohorts, tiles, n_tiles, grid, st, prof, split, ins);
}

}  // namespace epi3
