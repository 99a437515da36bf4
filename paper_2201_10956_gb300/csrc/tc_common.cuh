// Pieces shared by the tensor-core scan kernels: PTX wrappers (mbarriers, bulk copies,
// tcgen05 fences), the 128B-swizzled operand layout, and the epilogue arithmetic on
// count + 1 (derived cells, the table-free K2 bound, exact counts).
#pragma once

#include "epi3_internal.cuh"

namespace epi3 {
namespace {

// Bound of every mbarrier wait: 2^31 SM cycles (about 1 s at the 2.07 GHz maximum clock,
// longer at lower clocks).  No legitimate wait comes close.  The bound is read from the SM's
// own cycle counter: a read of the global timer costs hundreds of cycles, which a wait that
// starts just before its barrier completes would add to the pipeline.
constexpr long long kWaitCycles = 1LL << 31;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity; false on timeout (kWaitCycles) or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t a, unsigned parity, volatile int* abort_flag) {
    if (mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(a, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kWaitCycles) return false;
        }
    }
}
// mbar_wait that adds the cycles it spent to *acc (role profiling, optional).
__device__ __forceinline__ bool mbar_wait_t(uint32_t a, unsigned parity, volatile int* abort_flag,
                                            unsigned long long* acc) {
    if (!acc) return mbar_wait(a, parity, abort_flag);
    const long long t0 = clock64();
    const bool r = mbar_wait(a, parity, abort_flag);
    *acc += (unsigned long long)(clock64() - t0);
    return r;
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, unsigned bytes,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}
// Warp-wide forms: the whole (converged) warp executes the instruction and elect.sync lets one
// lane issue it.  tcgen05.mma / commit and bulk copies take their operands in uniform registers:
// issued by one lane inside a divergent branch, each costs an operand conversion that measured
// about 69 cycles per MMA on GB300 (48 cycles for an M=128 N=64 MMA issued warp-wide, which is
// its shared-memory operand read at 128 B/clk).  elect.sync picks the same leader every time in a
// full warp, so a commit covers the MMAs that the same lane issued.
__device__ __forceinline__ void mbar_arrive_tx_elect(uint32_t a, unsigned bytes) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}\n"
        ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s_elect(uint32_t dst, const void* src, unsigned bytes,
                                               uint32_t mbar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n}\n"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_commit_elect(uint32_t mbar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
        ::"r"(mbar) : "memory");
}
// A value every lane holds alike, made provably warp-uniform for the compiler.
__device__ __forceinline__ int warp_uniform(int v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ long long warp_uniform(long long v) {
    return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ void tc_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128B swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Byte offset of 16-byte unit u of row r in a 128-row, 128 B-per-row 128B-swizzled tile.
__host__ __device__ __forceinline__ uint32_t sw128_off(uint32_t r, uint32_t u) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((u ^ (r & 7u)) << 4);
}

// 8 bits -> 8 E2M1 nibbles (1.0 = 0x2) or 0; bit t lands in nibble t (low nibble first).
__device__ __forceinline__ uint32_t byte_to_e2m1(uint32_t b) {
    uint32_t x = b & 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x << 1;
}

// Position in a ring of n stages: stage index and the parity of the current pass.
struct Ring {
    int s;
    uint32_t ph;
};
__device__ __forceinline__ void ring_next(Ring& r, int n) {
    if (++r.s == n) {
        r.s = 0;
        r.ph ^= 1u;
    }
}

// ------------------------------------------------------------------ epilogue arithmetic
// Every class carries one extra "bias" sample (position N_c, one-hot 1 in every row of every
// SNP), so each accumulator holds u = count + 1.  The epilogue works on u throughout: the
// Stirling terms below need exactly count + 1, and an empty class reads as u = 1.  All values
// are integers below 2^24, so every float add and subtract here is exact.

// x + off as FP32, exact for 0 <= x < 2^23 and small off (x lands in the mantissa of 2^23).
__device__ __forceinline__ float count_plus(int x, float off) {
    return __fsub_rn(__int_as_float(x | 0x4B000000), 8388608.0f - off);
}

// Per (i, j) row of a tile and class: the constants of the derived cells, each + 3 (two
// u-values of count + 1 are subtracted from a count + 1).
struct RowCells {
    float xy[4];      // #(X = a, Y = b) + 3, index 2a + b
    float xa2[2];     // #(X = a, Y = 2) + 3
    float x2b[2];     // #(X = 2, Y = b) + 3
    float c22;        // #(X = 2, Y = 2) + 3
};

__device__ __forceinline__ RowCells row_cells(int4 pxy, int2 mx, int2 my, int nc) {
    RowCells rc;
    const int xa2_0 = mx.x - pxy.x - pxy.y, xa2_1 = mx.y - pxy.z - pxy.w;
    const int x2b_0 = my.x - pxy.x - pxy.z, x2b_1 = my.y - pxy.y - pxy.w;
    rc.xy[0] = count_plus(pxy.x, 3.f);
    rc.xy[1] = count_plus(pxy.y, 3.f);
    rc.xy[2] = count_plus(pxy.z, 3.f);
    rc.xy[3] = count_plus(pxy.w, 3.f);
    rc.xa2[0] = count_plus(xa2_0, 3.f);
    rc.xa2[1] = count_plus(xa2_1, 3.f);
    rc.x2b[0] = count_plus(x2b_0, 3.f);
    rc.x2b[1] = count_plus(x2b_1, 3.f);
    rc.c22 = count_plus(nc - mx.x - mx.y - x2b_0 - x2b_1, 3.f);
    return rc;
}

// u[9 gX + 3 gY + gZ] = cell count + 1 of one class, from the 8 accumulated cells
// n8[4a + 2b + z] (already + 1) and the FP32 copies of the pair tables (X, Z), (Y, Z) (each
// entry + 3) and of the marginal of Z (+ 9): the inclusion-exclusion of derive27 with every
// term shifted by one.
__device__ __forceinline__ void cells_u(const float* n8, const RowCells& rc, float4 pxz, float4 pyz,
                                        float2 mz9, float* u) {
    const float xz[2][2] = {{pxz.x, pxz.y}, {pxz.z, pxz.w}};
    const float yz[2][2] = {{pyz.x, pyz.y}, {pyz.z, pyz.w}};
    // #(X = 2, Z = z) + 3 = (#(Z = z) + 9) - (#(X=0, Z=z) + 3) - (#(X=1, Z=z) + 3)
    const float z2[2] = {__fsub_rn(__fsub_rn(mz9.x, xz[0][0]), xz[1][0]),
                         __fsub_rn(__fsub_rn(mz9.y, xz[0][1]), xz[1][1])};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float c0 = n8[4 * a + 2 * b], c1 = n8[4 * a + 2 * b + 1];
            u[9 * a + 3 * b] = c0;
            u[9 * a + 3 * b + 1] = c1;
            u[9 * a + 3 * b + 2] = __fsub_rn(__fsub_rn(rc.xy[2 * a + b], c0), c1);       // (a,b,2)
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int z = 0; z < 2; ++z)                                                       // (a,2,z)
            u[9 * a + 6 + z] = __fsub_rn(__fsub_rn(xz[a][z], u[9 * a + z]), u[9 * a + 3 + z]);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int z = 0; z < 2; ++z)                                                       // (2,b,z)
            u[18 + 3 * b + z] = __fsub_rn(__fsub_rn(yz[b][z], u[3 * b + z]), u[9 + 3 * b + z]);
#pragma unroll
    for (int a = 0; a < 2; ++a)                                                           // (a,2,2)
        u[9 * a + 8] = __fsub_rn(__fsub_rn(rc.xa2[a], u[9 * a + 6]), u[9 * a + 7]);
#pragma unroll
    for (int b = 0; b < 2; ++b)                                                           // (2,b,2)
        u[18 + 3 * b + 2] = __fsub_rn(__fsub_rn(rc.x2b[b], u[18 + 3 * b]), u[18 + 3 * b + 1]);
#pragma unroll
    for (int z = 0; z < 2; ++z)                                                           // (2,2,z)
        u[24 + z] = __fsub_rn(__fsub_rn(z2[z], u[18 + z]), u[21 + z]);
    u[26] = __fsub_rn(__fsub_rn(rc.c22, u[24]), u[25]);                                   // (2,2,2)
}

// The table-free K2 approximation (Stirling's form, lg2_hw) on u = count + 1: phi(n) =
// (u - 1/2) lg2(u), and the cell sum's argument is u0 + u1 = r + 2, so no conversion is
// needed; two interleaved FMA chains (cells 0..13 and 14..26) joined by one add.
__device__ __forceinline__ float k2_bound_u(const float* u0, const float* u1) {
    float acc[2] = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < kCells; ++q) {
        float& a = acc[q < 14 ? 0 : 1];
        const float us = __fadd_rn(u0[q], u1[q]);
        a = __fmaf_rn(__fsub_rn(us, 0.5f), lg2_hw(us), a);
        a = __fmaf_rn(-__fsub_rn(u0[q], 0.5f), lg2_hw(u0[q]), a);
        a = __fmaf_rn(-__fsub_rn(u1[q], 0.5f), lg2_hw(u1[q]), a);
    }
    return __fmaf_rn(0.6931471805599453f, __fadd_rn(acc[0], acc[1]), -27.f * 0.9189385332046727f);
}

// k2_bound_u of two tables at once (four independent chains), for the register-split form.
__device__ __forceinline__ void k2_bound_u2(const float* u0a, const float* u1a, const float* u0b,
                                            const float* u1b, float* out) {
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int q = 0; q < kCells; ++q) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float x0 = t ? u0b[q] : u0a[q], x1 = t ? u1b[q] : u1a[q];
            float& a = acc[t][q < 14 ? 0 : 1];
            const float us = __fadd_rn(x0, x1);
            a = __fmaf_rn(__fsub_rn(us, 0.5f), lg2_hw(us), a);
            a = __fmaf_rn(-__fsub_rn(x0, 0.5f), lg2_hw(x0), a);
            a = __fmaf_rn(-__fsub_rn(x1, 0.5f), lg2_hw(x1), a);
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
        out[t] = __fmaf_rn(0.6931471805599453f, __fadd_rn(acc[t][0], acc[t][1]),
                           -27.f * 0.9189385332046727f);
}

// Two FP32 lanes per 64-bit register (two tables at once): the f32x2 instructions of sm_100 and
// later round each lane exactly like the scalar __fadd_rn / __fsub_rn / __fmaf_rn, so every lane
// equals the scalar code's result bit for bit.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y, r;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " add.rn.f32x2 r, x, y;\n mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y, r;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " sub.rn.f32x2 r, x, y;\n mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 x, y, z, r;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " mov.b64 z, {%6, %7};\n fma.rn.f32x2 r, x, y, z;\n mov.b64 {%0, %1}, r;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 f2_dup(float a) { return make_float2(a, a); }

// Lane arithmetic for the bound of one table (float) or two tables at once (float2, f32x2
// instructions): every lane rounds like the scalar __fadd_rn / __fsub_rn / __fmaf_rn.
struct LaneOps1 {
    typedef float T;
    static __device__ __forceinline__ T add(T a, T b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ T lg(T a) { return lg2_hw(a); }
    static __device__ __forceinline__ T dup(float a) { return a; }
};
struct LaneOps2 {
    typedef float2 T;
    static __device__ __forceinline__ T add(T a, T b) { return f2_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return f2_sub(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return f2_fma(a, b, c); }
    static __device__ __forceinline__ T lg(T a) { return make_float2(lg2_hw(a.x), lg2_hw(a.y)); }
    static __device__ __forceinline__ T dup(float a) { return f2_dup(a); }
};

// The table-free bound (k2_bound_u's terms) with both classes' cells derived on the fly (the
// operations of cells_u, per class), each cell's three terms chained as soon as both classes'
// values are known: no 27-cell array is ever live.  n8[c][4 a + 2 b + z] = count + 1 of the
// counted cells, xz[c][a][z] / yz[c][b][z] = pair-table entries + 3, mz[c][z] = marginal of Z
// + 9, rc[c] = the row cells of class c.  Cells enter the two chains in derivation order; the
// bound's error analysis (every finished cell adds a positive amount; 82 roundings of at most
// 2^-24 of the largest partial sum) holds for any order.
template <class L>
__device__ __forceinline__ typename L::T k2_bound_cells(const typename L::T (*n8)[8],
                                                        const RowCells* rc,
                                                        const typename L::T (*xz)[2][2],
                                                        const typename L::T (*yz)[2][2],
                                                        const typename L::T (*mz)[2]) {
    typedef typename L::T T;
    T acc[2] = {L::dup(0.f), L::dup(0.f)};
    const T half = L::dup(0.5f);
    auto term = [&](int q, T u0, T u1) {
        T& a = acc[q & 1];
        const T us = L::add(u0, u1);
        a = L::fma(L::sub(us, half), L::lg(us), a);
        a = L::fma(L::sub(half, u0), L::lg(u0), a);
        a = L::fma(L::sub(half, u1), L::lg(u1), a);
    };
    auto d2 = [&](T x, T y, T z) { return L::sub(L::sub(x, y), z); };
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int e = 4 * a + 2 * b;
            term(9 * a + 3 * b, n8[0][e], n8[1][e]);
            term(9 * a + 3 * b + 1, n8[0][e + 1], n8[1][e + 1]);
            term(9 * a + 3 * b + 2, d2(L::dup(rc[0].xy[2 * a + b]), n8[0][e], n8[0][e + 1]),
                 d2(L::dup(rc[1].xy[2 * a + b]), n8[1][e], n8[1][e + 1]));
        }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        T a2z[2][2];  // [class][z]
#pragma unroll
        for (int z = 0; z < 2; ++z) {
#pragma unroll
            for (int c = 0; c < 2; ++c) a2z[c][z] = d2(xz[c][a][z], n8[c][4 * a + z], n8[c][4 * a + 2 + z]);
            term(9 * a + 6 + z, a2z[0][z], a2z[1][z]);
        }
        term(9 * a + 8, d2(L::dup(rc[0].xa2[a]), a2z[0][0], a2z[0][1]),
             d2(L::dup(rc[1].xa2[a]), a2z[1][0], a2z[1][1]));
    }
    T c2bz[2][2][2];  // [class][b][z]
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
        for (int z = 0; z < 2; ++z) {
#pragma unroll
            for (int c = 0; c < 2; ++c) c2bz[c][b][z] = d2(yz[c][b][z], n8[c][2 * b + z], n8[c][4 + 2 * b + z]);
            term(18 + 3 * b + z, c2bz[0][b][z], c2bz[1][b][z]);
        }
        term(18 + 3 * b + 2, d2(L::dup(rc[0].x2b[b]), c2bz[0][b][0], c2bz[0][b][1]),
             d2(L::dup(rc[1].x2b[b]), c2bz[1][b][0], c2bz[1][b][1]));
    }
    T c22z[2][2];  // [class][z]
#pragma unroll
    for (int z = 0; z < 2; ++z) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const T z2 = d2(mz[c][z], xz[c][0][z], xz[c][1][z]);   // #(X = 2, Z = z) + 3
            c22z[c][z] = d2(z2, c2bz[c][0][z], c2bz[c][1][z]);
        }
        term(24 + z, c22z[0][z], c22z[1][z]);
    }
    term(26, d2(L::dup(rc[0].c22), c22z[0][0], c22z[0][1]), d2(L::dup(rc[1].c22), c22z[1][0], c22z[1][1]));
    return L::add(acc[0], acc[1]);  // in log2 units, before the final scale and offset
}
__device__ __forceinline__ float k2_bound_finish(float s) {
    return __fmaf_rn(0.6931471805599453f, s, -27.f * 0.9189385332046727f);
}

// Exact integer cells r = u - 1 of both classes; false unless every cell lies in [0, N_c]
// (which keeps every log-factorial lookup of the table in range).
__device__ __forceinline__ bool counts_of(const float* u0, const float* u1, int n0, int n1,
                                          int* r0, int* r1) {
    bool ok = true;
#pragma unroll
    for (int q = 0; q < kCells; ++q) {
        // u + 2^23 - 1 holds u - 1 in its mantissa for 1 <= u < 2^23; anything else falls
        // outside [0, N_c]
        r0[q] = __float_as_int(__fadd_rn(u0[q], 8388607.0f)) - 0x4B000000;
        r1[q] = __float_as_int(__fadd_rn(u1[q], 8388607.0f)) - 0x4B000000;
        ok = ok && (unsigned)r0[q] <= (unsigned)n0 && (unsigned)r1[q] <= (unsigned)n1;
    }
    return ok;
}



// ------------------------------------------------------------------ candidate stage
// Named barrier 1 over the epilogue threads (kThreads of them); the variant also returns
// whether any of them passed true.
template <int kThreads>
__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}
template <int kThreads>
__device__ __forceinline__ bool epi_sync_or(bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, 1, %2, a;\n"
        " selp.u32 %0, 1, 0, b;\n}\n"
        : "=r"(r) : "r"((uint32_t)p), "n"(kThreads) : "memory");
    return r != 0;
}

constexpr int kCandCap = 1024;               // per-CTA candidate buffer (power of two)
constexpr int kPruneAt = kCandCap / 2;       // local candidates that trigger a prune

template <int kThreads>
__device__ void sort_cands(Cand* buf, int tid) {
    for (int size = 2; size <= kCandCap; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < kCandCap / 2; t += kThreads) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const Cand x = buf[lo], y = buf[hi];
                if ((x.s > y.s) == up) {
                    buf[lo] = y;
                    buf[hi] = x;
                }
            }
            epi_sync<kThreads>();
        }
}

struct EpiShared {
    Cand buf[kCandCap];
    int cnt, keep;
    float tloc;
};

// Sort the buffer (cnt <= kCandCap entries), publish this CTA's band threshold, keep the
// entries inside the band; spill to the global list when too many tie.  Called by all
// epilogue threads.
template <int kThreads>
__device__ int epi_prune(const CohortDev& a, EpiShared& es, int cnt, int tid, bool final_flush) {
    const float kInf = __int_as_float(0x7f800000);
    if (cnt >= a.top_k) {
        for (int idx = cnt + tid; idx < kCandCap; idx += kThreads) es.buf[idx].s = kInf;
        epi_sync<kThreads>();
        sort_cands<kThreads>(es.buf, tid);
        if (tid == 0) {
            const float tl = band_threshold(es.buf[a.top_k - 1].s, a.k2.rel, a.k2.abs_);
            atomicMin(&a.ctrl->thr, __float_as_uint(tl));
            es.tloc = fminf(es.tloc, tl);
        }
    }
    if (tid == 0) es.keep = 0;
    epi_sync<kThreads>();
    const float t = fminf(es.tloc, __uint_as_float(*(volatile unsigned*)&a.ctrl->thr));
    if (final_flush || cnt < a.top_k) {
        for (int idx = tid; idx < cnt; idx += kThreads) {
            const Cand e = es.buf[idx];
            if (e.s <= t) {
                const unsigned pos = atomicAdd(&a.ctrl->n_cand, 1u);
                if (pos < (unsigned long long)a.cand_cap) a.cand[pos] = e;
                else atomicOr(&a.ctrl->status, kStCandOverflow);
            }
        }
        epi_sync<kThreads>();
        return 0;
    }
    int keep = 0;
    for (int idx = tid; idx < cnt; idx += kThreads) keep += (es.buf[idx].s <= t);
    if (keep) atomicAdd(&es.keep, keep);
    epi_sync<kThreads>();
    int kept = es.keep;
    if (kept > kPruneAt) {
        for (int idx = tid; idx < kept; idx += kThreads) {
            const Cand e = es.buf[idx];
            const unsigned pos = atomicAdd(&a.ctrl->n_cand, 1u);
            if (pos < (unsigned long long)a.cand_cap) a.cand[pos] = e;
            else atomicOr(&a.ctrl->status, kStCandOverflow);
        }
        kept = 0;
    }
    epi_sync<kThreads>();
    return kept;
}

// A candidate straight to the cohort's global list (the local buffer is full).
__device__ __forceinline__ void cand_global(const CohortDev& a, const Cand& e) {
    const unsigned pos = atomicAdd(&a.ctrl->n_cand, 1u);
    if (pos < (unsigned long long)a.cand_cap) a.cand[pos] = e;
    else atomicOr(&a.ctrl->status, kStCandOverflow);
}

}  // namespace
}  // namespace epi3
