// Host side of the C ABI (include/epi3.h): handles, validation, device memory, the
// scan's launch sequence, error reporting and statistics.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <chrono>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "epi3_internal.cuh"

using namespace epi3;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(EPI3_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(EPI3_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Fault injection for tests of the error paths, all without faulting the GPU:
// EPI3_FAULT=alloc makes device allocations fail, EPI3_FAULT=launch makes scan launches fail,
// EPI3_FAULT=timeout makes the tensor-core scan's MMA issuer wait on a barrier nobody
// signals, so its bounded wait runs out (1 s) and the scan returns EPI3_ERR_TIMEOUT;
// EPI3_FAULT=cand starts a handle with a 128-entry candidate list, so scans overflow it and
// take the retry path with a larger list.
bool inject(const char* what) {
    const char* f = getenv("EPI3_FAULT");
    return f && strcmp(f, what) == 0;
}

// Device memory of handles and batches.  Freed blocks are kept in a per-process cache (per
// device, at most EPI3_CACHE_MB megabytes, default 4096; 0 turns the cache off) and handed to
// later allocations of up to their size, so that creating and destroying handles per data set
// does not pay cudaMalloc and cudaFree each time.  A block enters the cache only after its
// device is synchronised, as cudaFree would do, so no queued kernel can still use it.  An
// allocation that fails while blocks are cached empties the cache and tries once more.
struct MemBlock {
    void* p;
    size_t bytes;
    int dev;
};
std::mutex g_mem_mu;
std::unordered_map<void*, MemBlock> g_mem_live;   // blocks handed out by dev_alloc
std::vector<MemBlock> g_mem_free;                 // cached blocks
size_t g_mem_free_bytes = 0;

size_t mem_cache_limit() {
    static const size_t lim = [] {
        const char* v = getenv("EPI3_CACHE_MB");
        long long mb = v ? atoll(v) : 4096;
        return (size_t)(mb < 0 ? 0 : mb) << 20;
    }();
    return lim;
}

void mem_drop_cache() {  // caller holds g_mem_mu
    int cur = 0;
    cudaGetDevice(&cur);
    for (const MemBlock& b : g_mem_free) {
        if (b.dev != cur) cudaSetDevice(b.dev);
        cudaFree(b.p);
        if (b.dev != cur) cudaSetDevice(cur);
    }
    g_mem_free.clear();
    g_mem_free_bytes = 0;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (inject("alloc")) return cudaErrorMemoryAllocation;
    bytes = (std::max(bytes, (size_t)16) + 255) & ~(size_t)255;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    // the smallest cached block of this device that holds the request without wasting more
    // than the request itself
    size_t best = (size_t)-1;
    for (size_t t = 0; t < g_mem_free.size(); ++t) {
        const MemBlock& b = g_mem_free[t];
        if (b.dev == dev && b.bytes >= bytes && b.bytes <= 2 * bytes &&
            (best == (size_t)-1 || b.bytes < g_mem_free[best].bytes))
            best = t;
    }
    if (best != (size_t)-1) {
        const MemBlock b = g_mem_free[best];
        g_mem_free[best] = g_mem_free.back();
        g_mem_free.pop_back();
        g_mem_free_bytes -= b.bytes;
        g_mem_live[b.p] = b;
        *p = b.p;
        return cudaSuccess;
    }
    e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation && !g_mem_free.empty()) {
        (void)cudaGetLastError();
        mem_drop_cache();
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    g_mem_live[*p] = MemBlock{*p, bytes, dev};
    return cudaSuccess;
}

// Release a block of dev_alloc (null is ignored; anything else goes to cudaFree).  `synced`:
// the caller has synchronised the only stream that used the block, so the device-wide
// synchronisation is skipped.
void dev_free(void* p, bool synced = false) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    const auto it = g_mem_live.find(p);
    if (it == g_mem_live.end()) {
        cudaFree(p);
        return;
    }
    const MemBlock b = it->second;
    g_mem_live.erase(it);
    const size_t lim = mem_cache_limit();
    if (b.bytes > lim) {
        cudaFree(p);
        return;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    if (b.dev != cur) cudaSetDevice(b.dev);
    // as cudaFree: no queued work still uses the block
    const cudaError_t e = synced ? cudaSuccess : cudaDeviceSynchronize();
    if (b.dev != cur) cudaSetDevice(cur);
    if (e != cudaSuccess) {   // a failed context: give the block back to the driver
        cudaFree(p);
        return;
    }
    while (g_mem_free_bytes + b.bytes > lim && !g_mem_free.empty()) {   // oldest first
        const MemBlock o = g_mem_free.front();
        g_mem_free.erase(g_mem_free.begin());
        g_mem_free_bytes -= o.bytes;
        if (o.dev != cur) cudaSetDevice(o.dev);
        cudaFree(o.p);
        if (o.dev != cur) cudaSetDevice(cur);
    }
    g_mem_free.push_back(b);
    g_mem_free_bytes += b.bytes;
}

// Pinned host buffers of handles and batches (status and result read-back), cached the same
// way: freed only after the stream that copied into them was synchronised.
std::unordered_map<void*, size_t> g_pin_live;
std::vector<std::pair<void*, size_t>> g_pin_free;
constexpr size_t kPinCacheMax = 256;   // cached blocks

cudaError_t host_alloc(void** p, size_t bytes) {
    *p = nullptr;
    bytes = (std::max(bytes, (size_t)16) + 255) & ~(size_t)255;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    for (size_t t = 0; t < g_pin_free.size(); ++t)
        if (g_pin_free[t].second >= bytes && g_pin_free[t].second <= 2 * bytes) {
            *p = g_pin_free[t].first;
            g_pin_live[*p] = g_pin_free[t].second;
            g_pin_free[t] = g_pin_free.back();
            g_pin_free.pop_back();
            return cudaSuccess;
        }
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    g_pin_live[*p] = bytes;
    return cudaSuccess;
}

void host_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mem_mu);
    const auto it = g_pin_live.find(p);
    if (it == g_pin_live.end() || mem_cache_limit() == 0 || g_pin_free.size() >= kPinCacheMax) {
        if (it != g_pin_live.end()) g_pin_live.erase(it);
        cudaFreeHost(p);
        return;
    }
    g_pin_free.emplace_back(p, it->second);
    g_pin_live.erase(it);
}

long long pairs(long long m) { return m < 2 ? 0 : m * (m - 1) / 2; }

// Triplets (i, j, k), k > j, of the pairs with index in [pb, pe) (p = j(j-1)/2 + i).
long long triplets_in_pairs(long long M, long long pb, long long pe) {
    long long t = 0;
    for (long long j = 1; j < M; ++j) {
        const long long lo = j * (j - 1) / 2, hi = lo + j;
        const long long a = pb > lo ? pb : lo, b = pe < hi ? pe : hi;
        if (b > a) t += (b - a) * (M - 1 - j);
    }
    return t;
}

}  // namespace

struct epi3_handle {
    int device = 0, sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int flags = 0;
    int M = 0, N = 0, N0 = 0, N1 = 0;
    Planes pl{};
    uint4* d_planes = nullptr;
    float2* d_lf2 = nullptr;
    double* d_lf64 = nullptr;
    K2Tables k2{};
    int g_bits = 0;
    double approx_err = 0.0;      // measured max |lf_approx - lf| over 0..N+1
    Ctrl* d_ctrl = nullptr;
    Cand* d_cand = nullptr;
    long long cand_cap = 0;
    Final* d_fin = nullptr;
    double* d_out_scores = nullptr;
    int* d_out_trip = nullptr;
    int4* d_pt = nullptr;         // pair tables (8-cell forms), built on first use
    void* d_pair_scratch = nullptr;  // pairwise scan: selection passes + outputs
    size_t pair_scratch_bytes = 0;
    int2* d_marg = nullptr;
    float4* d_ptf = nullptr;         // tensor scan: pair tables + 3 as FP32
    float2* d_margf = nullptr;       // tensor scan: marginals + 9 as FP32
    PairTables ptab{};
    uint8_t* d_oh = nullptr;      // pre-tiled one-hot operand of the tensor-core form
    int oh_kind = -1;             // element kind d_oh was built for (kKind*, -1: none)
    int oh_ks[2] = {0, 0};
    long long oh_off1 = 0;
    float* dbg = nullptr;         // device buffer of epi3_scan_scores (during that call only)
    unsigned long long* tsum = nullptr;  // checksum slots of epi3_scan_checksum (that call only)
    CohortDev* d_cd = nullptr;    // this data set's descriptor for the tensor-core kernel
    bool profile = false;
    int mma_form = 0;                    // tensor scan: 0 = measured (tuner), 1 = plain, 2 = split
    int tuned_path = 0;                  // path "auto": the tuner's choice (0 = not yet measured)
    int tuned_form = 0;                  // the tuner's tensor-scan form (1 plain, 2 split)
    int tuned_form_path = 0;             // ... for this tensor path
    bool autotune = true;                // option "autotune"
    bool tuning = false;                 // a tuning scan is running
    // last compacted-form scan: its plan's work terms and (tuning scans) compaction time
    double last_cmp_chunks = 0.0, last_cmp_steps = 0.0;
    float last_compact_ms = 0.f;
    std::vector<cudaEvent_t> cmp_ev;     // event pairs around the compaction launches
    unsigned long long* d_prof = nullptr;
    uint8_t* d_cmp = nullptr;     // compacted chunks of the sample-compacted tensor form
    size_t cmp_bytes = 0;
    size_t cmp_cap = (size_t)2 << 30;  // option "cmp_buffer_mb": bytes of compacted chunks at once
    CmpFirst* d_firsts = nullptr; // per first SNP: chunk bases, K-steps, tiles
    std::vector<int2> h_marg;     // marginals on the host (the compacted sets' sizes)
    int4* d_tiles = nullptr;      // tile list of the tensor-core form
    long long n_tiles = 0, tiles_pb = -1, tiles_pe = -1;
    Ctrl* h_ctrl = nullptr;       // pinned
    double* h_scores = nullptr;   // pinned [EPI3_MAX_TOPK]
    int* h_trip = nullptr;        // pinned [EPI3_MAX_TOPK * 3]
    int path = EPI3_PATH_AUTO;          // scan path (option "path"); auto = E2M1 tensor form
    int threads = 128;
    int ctas_per_sm = 0;
    bool timing = false;
    // scan start, kernels start, kernels end, scan end
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    epi3_stats stats{};
};

namespace {

void release(epi3_handle* h) {
    if (!h) return;
    // every buffer of the handle is used on its stream only: once that is synchronised
    // the blocks go to the cache without a device-wide synchronisation
    const bool synced = h->stream && cudaStreamSynchronize(h->stream) == cudaSuccess;
    dev_free(h->d_planes, synced);
    dev_free(h->d_lf2, synced);
    dev_free(h->d_lf64, synced);
    dev_free(h->d_ctrl, synced);
    dev_free(h->d_cand, synced);
    dev_free(h->d_fin, synced);
    dev_free(h->d_out_scores, synced);
    dev_free(h->d_out_trip, synced);
    dev_free(h->d_pt, synced);
    dev_free(h->d_pair_scratch, synced);
    dev_free(h->d_marg, synced);
    dev_free(h->d_ptf, synced);
    dev_free(h->d_margf, synced);
    dev_free(h->d_oh, synced);
    dev_free(h->d_cmp, synced);
    dev_free(h->d_firsts, synced);
    dev_free(h->d_tiles, synced);
    dev_free(h->d_cd, synced);
    dev_free(h->d_prof, synced);
    host_free(h->h_ctrl);
    host_free(h->h_scores);
    host_free(h->h_trip);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->cmp_ev) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int check_device(int* dev, int* sms) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0)
        return fail(EPI3_ERR_UNSUPPORTED, "no CUDA device (%s)",
                    e == cudaSuccess ? "count 0" : cudaGetErrorString(e));
    CK(cudaGetDevice(dev), "cudaGetDevice");
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, *dev), "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
        return fail(EPI3_ERR_UNSUPPORTED, "device %d is sm_%d%d; this build targets sm_103a only",
                    *dev, prop.major, prop.minor);
    *sms = prop.multiProcessorCount;
    return EPI3_OK;
}

// Log-factorial tables of Eq. 1.  lf[n] = lf[n-1] + log(n) in FP64 (the same additions
// in the same order as summing log b for b = 1..n).  The FP32 pair splits lf = hi + lo
// with hi on the grid 2^-g, g the largest integer with lf[N+1] * 2^g < 2^23, so that
// every hi difference and partial sum in k2_f32 is exact.
int build_k2_tables(epi3_handle* h) {
    const int n = h->N + 2;
    std::vector<double> lf(n);
    lf[0] = 0.0;
    for (int i = 1; i < n; ++i) lf[i] = lf[i - 1] + std::log((double)i);
    int e = 0;
    std::frexp(lf[n - 1], &e);  // lf[N+1] < 2^e
    const int g = 23 - e;
    std::vector<float2> lf2(n);
    for (int i = 0; i < n; ++i) {
        const double hi = std::ldexp(std::nearbyint(std::ldexp(lf[i], g)), -g);
        lf2[i].x = (float)hi;
        lf2[i].y = (float)(lf[i] - hi);
    }
    h->g_bits = g;
    CK(dev_alloc((void**)&h->d_lf64, sizeof(double) * n), "alloc lf64");
    CK(dev_alloc((void**)&h->d_lf2, sizeof(float2) * n), "alloc lf2");
    CK(cudaMemcpyAsync(h->d_lf64, lf.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream),
       "upload lf64");
    CK(cudaMemcpyAsync(h->d_lf2, lf2.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, h->stream),
       "upload lf2");
    h->k2.lf2 = h->d_lf2;
    h->k2.lf64 = h->d_lf64;
    h->k2.rel = std::ldexp(1.0f, -23);
    h->k2.abs_ = std::ldexp(1.0f, -(g + 13));
    // Pruning bound of the tensor scan: |K2 bound - s32| for any table of this data set.
    //   delta  measured max of (n + 1/2) |lg2_hw(n+1) - log2(n+1)| over n = 0..N+1
    //   Stirling remainders: at most 1/6 per cell (e(r+1) - e(r0) - e(r1), 0 < e <= 1/12)
    //   FMA chains (81 steps in two chains over disjoint cells, then one add; log2 units):
    //     each of the 82 roundings is at most 2^-24 |acc|; every finished cell adds a positive
    //     amount (its K2 term + ln(2 pi)/2 - Stirling remainder), so every partial sum obeys
    //     0 <= acc <= (K + 27 (ln(2 pi)/2 + 1/12)) / ln2 + T + 81 delta, with K = 27 ln(N+2)
    //     + N ln 2 bounding K2 and T = (N + 3/2) log2(N + 2) the largest single product
    //   final FMA and the FP32 constants: 2^-22 (K + 27 ln(2 pi)/2 + ln2 (K/ln2 + T))
    //   s32 against K2: rel * K + abs
    // and the bound used is twice the sum plus 1/2 nat.
    double* d_err = nullptr;
    CK(dev_alloc((void**)&d_err, sizeof(double)), "alloc approx error");
    double delta = 0.0;
    cudaError_t ce = launch_approx_error(h->d_lf64, n, d_err, h->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&delta, d_err, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    dev_free(d_err);
    CK(ce, "approx error");
    const double u = std::ldexp(1.0, -24), ln2 = std::log(2.0);
    const double kmax = 27.0 * std::log((double)h->N + 2.0) + (double)h->N * ln2;
    const double tmax = ((double)h->N + 1.5) * std::log2((double)h->N + 2.0);
    const double amax = (kmax + 27.0 * (0.9189385332046727 + 1.0 / 12.0)) / ln2 + tmax +
                        81.0 * delta;
    const double d_approx = 27.0 / 6.0 + ln2 * (81.0 * delta + 82.0 * u * amax) +
                            4.0 * u * (kmax + 27.0 * 0.9189385332046727 + ln2 * amax);
    const double d_s32 = (double)h->k2.rel * kmax + (double)h->k2.abs_;
    h->k2.prune_delta = (float)(2.0 * (d_approx + d_s32) + 0.5);
    h->approx_err = delta;
    h->stats.k2_rel_bound = h->k2.rel;
    h->stats.k2_abs_bound = h->k2.abs_;
    h->stats.k2_prune_bound = h->k2.prune_delta;
    return EPI3_OK;
}

int create_impl(epi3_handle* h, const uint8_t* geno, const uint8_t* pheno) {
    const size_t MN = (size_t)h->M * h->N;
    uint8_t* d_geno = nullptr;
    uint8_t* d_pheno = nullptr;
    int* d_counts = nullptr;
    int rc = EPI3_OK;
    bool synced = false;   // the stream that used the temporaries has been synchronised
    auto cleanup = [&]() {
        if (!(h->flags & EPI3_DEVICE_PTRS)) {
            dev_free(d_geno, synced);
            dev_free(d_pheno, synced);
        }
        dev_free(d_counts, synced);
    };
    do {
        cudaError_t e;
        if ((e = dev_alloc((void**)&h->d_ctrl, sizeof(Ctrl))) != cudaSuccess) { rc = cuda_fail(e, "alloc ctrl"); break; }
        if ((e = host_alloc((void**)&h->h_ctrl, sizeof(Ctrl))) != cudaSuccess) { rc = cuda_fail(e, "pinned ctrl"); break; }
        if (h->flags & EPI3_DEVICE_PTRS) {
            d_geno = const_cast<uint8_t*>(geno);
            d_pheno = const_cast<uint8_t*>(pheno);
        } else {
            if ((e = dev_alloc((void**)&d_geno, MN)) != cudaSuccess) { rc = cuda_fail(e, "alloc genotypes"); break; }
            if ((e = dev_alloc((void**)&d_pheno, h->N)) != cudaSuccess) { rc = cuda_fail(e, "alloc phenotype"); break; }
            if ((e = cudaMemcpyAsync(d_geno, geno, MN, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "copy genotypes"); break; }
            if ((e = cudaMemcpyAsync(d_pheno, pheno, h->N, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "copy phenotype"); break; }
        }
        if ((e = dev_alloc((void**)&d_counts, sizeof(int) * class_counts_len(h->N))) != cudaSuccess) { rc = cuda_fail(e, "alloc counts"); break; }
        if ((e = launch_reset(h->d_ctrl, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "reset"); break; }
        if ((e = launch_class_index(d_pheno, h->N, d_counts, h->d_ctrl, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "class_index launch"); break; }
        int counts[2] = {0, 0};
        if (!(h->flags & EPI3_DEVICE_PTRS)) {
            // host inputs: the class sizes come from the phenotype on the host, while the copies
            // and the class index run (no wait for the device here)
            int n1 = 0;
            bool bad = false;
            for (int t = 0; t < h->N; ++t) {
                n1 += pheno[t] == 1;
                bad |= pheno[t] > 1;
            }
            if (bad) { rc = fail(EPI3_ERR_ARG, "phenotype value > 1"); break; }
            counts[0] = h->N - n1;
            counts[1] = n1;
        } else {
            if ((e = cudaMemcpyAsync(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read counts"); break; }
            if ((e = cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read status"); break; }
            if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = cuda_fail(e, "class_index"); break; }
            if (h->h_ctrl->status & kStBadPhenotype) { rc = fail(EPI3_ERR_ARG, "phenotype value > 1"); break; }
        }
        h->N0 = counts[0];
        h->N1 = counts[1];
        Planes& pl = h->pl;
        pl.M = h->M;
        pl.W4[0] = (h->N0 + kSamplesPerGroup - 1) / kSamplesPerGroup;
        pl.W4[1] = (h->N1 + kSamplesPerGroup - 1) / kSamplesPerGroup;
        pl.coff[0] = 0;
        pl.coff[1] = 2LL * pl.W4[0] * h->M;
        pl.pad[0] = kSamplesPerGroup * pl.W4[0] - h->N0;
        pl.pad[1] = kSamplesPerGroup * pl.W4[1] - h->N1;
        const size_t n4 = 2ull * (pl.W4[0] + pl.W4[1]) * h->M;
        if ((e = dev_alloc((void**)&h->d_planes, n4 * sizeof(uint4))) != cudaSuccess) { rc = cuda_fail(e, "alloc planes"); break; }
        pl.planes = h->d_planes;
        if ((e = cudaEventRecord(h->ev[0], h->stream)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
        if ((e = launch_pack(d_geno, d_pheno, h->M, h->N, d_counts, h->N0, h->N1, pl, h->d_planes, h->d_ctrl, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "pack launch"); break; }
        if ((e = cudaEventRecord(h->ev[1], h->stream)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
        if ((e = cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read status"); break; }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = cuda_fail(e, "pack"); break; }
        synced = true;
        if (h->h_ctrl->status & (kStBadGenotype | kStBadPhenotype)) {
            rc = fail(EPI3_ERR_ARG, (h->h_ctrl->status & kStBadGenotype) ? "genotype value > 2"
                                                                            : "phenotype value > 1");
            break;
        }
        cudaEventElapsedTime(&h->stats.pack_ms, h->ev[0], h->ev[1]);
    } while (0);
    cleanup();
    if (rc != EPI3_OK) return rc;
    if ((rc = build_k2_tables(h)) != EPI3_OK) return rc;
    // FP32 candidate list: the CTAs flush their in-band candidates before the shared threshold
    // tightens, about 10^5 of them on a scan that fills the GPU (a list that overflows costs a
    // whole rescan, in a batch a second replay of every cohort)
    const long long m = h->M;
    h->cand_cap = inject("cand") ? 128 : m * (m - 1) * (m - 2) / 6 >= (1LL << 22) ? 1LL << 20 : 1LL << 16;
    CK(dev_alloc((void**)&h->d_cand, sizeof(Cand) * h->cand_cap), "alloc candidates");
    CK(dev_alloc((void**)&h->d_fin, sizeof(Final) * kFinalCap), "alloc final");
    CK(dev_alloc((void**)&h->d_out_scores, sizeof(double) * EPI3_MAX_TOPK), "alloc out scores");
    CK(dev_alloc((void**)&h->d_out_trip, sizeof(int) * 3 * EPI3_MAX_TOPK), "alloc out triplets");
    CK(host_alloc((void**)&h->h_scores, sizeof(double) * EPI3_MAX_TOPK), "pinned scores");
    CK(host_alloc((void**)&h->h_trip, sizeof(int) * 3 * EPI3_MAX_TOPK), "pinned triplets");
    return EPI3_OK;
}

// Pair tables and marginals of the 8-cell forms (built once per handle).
int ensure_pair_tables(epi3_handle* h) {
    if (h->d_pt) return EPI3_OK;
    const long long np = pairs(h->M);
    CK(dev_alloc((void**)&h->d_pt, sizeof(int4) * 2 * (size_t)np), "alloc pair tables");
    CK(dev_alloc((void**)&h->d_marg, sizeof(int2) * 2 * (size_t)h->M), "alloc marginals");
    // stream-ordered: every consumer runs on the handle's stream (the host reads the marginals
    // after synchronising it)
    CK(launch_pair_tables(h->pl, h->d_pt, h->d_marg, np, h->stream), "pair tables launch");
    h->ptab.pt = h->d_pt;
    h->ptab.marg = h->d_marg;
    h->ptab.n_pairs = np;
    h->ptab.n_c[0] = h->N0;
    h->ptab.n_c[1] = h->N1;
    return EPI3_OK;
}

// Tensor-core form: pre-tiled one-hot operand (built once per element type).
int ensure_pair_floats(epi3_handle* h) {
    if (!h->d_ptf) {  // the tensor scans' FP32 copies of the pair tables (built once)
        const long long np = h->ptab.n_pairs;
        CK(dev_alloc((void**)&h->d_ptf, sizeof(float4) * 2 * (size_t)np), "alloc FP32 pair tables");
        CK(dev_alloc((void**)&h->d_margf, sizeof(float2) * 2 * (size_t)h->M), "alloc FP32 marginals");
        CK(launch_pair_floats(h->d_pt, h->d_marg, np, h->M, h->d_ptf, h->d_margf, h->stream),
           "FP32 pair tables launch");
        h->ptab.ptf = h->d_ptf;
        h->ptab.margf = h->d_margf;
    }
    return EPI3_OK;
}

int ensure_onehot(epi3_handle* h, int kind) {
    const int rc = ensure_pair_floats(h);
    if (rc != EPI3_OK) return rc;
    if (h->d_oh && h->oh_kind == kind) return EPI3_OK;
    dev_free(h->d_oh);
    h->d_oh = nullptr;
    const int spk = mma_samples_per_step(kind);
    // N_c samples plus the bias sample (position N_c) of a non-empty class
    const int ks0 = h->N0 ? h->N0 / spk + 1 : 0, ks1 = h->N1 ? h->N1 / spk + 1 : 0;
    const int kbc = (h->M + 63) / 64;
    CK(dev_alloc((void**)&h->d_oh, onehot_bytes(h->M, ks0, ks1)), "alloc one-hot operand");
    h->oh_ks[0] = ks0;
    h->oh_ks[1] = ks1;
    h->oh_off1 = (long long)kbc * ks0;
    CK(launch_onehot(h->pl, h->d_oh, h->oh_off1, ks0, ks1, kbc, kind, h->stream), "one-hot launch");
    uint8_t* yoh = h->d_oh + (size_t)kbc * (ks0 + ks1) * 16384;
    uint8_t* xoh = yoh + (size_t)2 * kbc * (ks0 + ks1) * 8192;
    CK(launch_onehot_views(h->d_oh, h->oh_off1, ks0, ks1, kbc, h->M, yoh, xoh, h->stream),
       "one-hot views launch");
    CK(cudaStreamSynchronize(h->stream), "one-hot");
    h->oh_kind = kind;
    return EPI3_OK;
}

// Tiles (i, 32-SNP block of j, 64-SNP block of k) holding a triplet i<j<k whose pair (i, j)
// lies in [pb, pe); third-SNP block outermost so concurrent CTAs share A chunks in L2.
void append_tiles(int M, long long pb, long long pe, int cohort, std::vector<int4>& t) {
    const int kbc = (M + 63) / 64, jbc = (M + 31) / 32;
    for (int kb = 0; kb < kbc; ++kb) {
        const int k_hi = std::min(64 * kb + 63, M - 1);
        for (int jb = 0; jb < jbc; ++jb) {
            const int j_lo = 32 * jb, j_hi = std::min(32 * jb + 31, M - 1);
            if (j_lo >= k_hi) continue;
            const int i_end = std::min(j_hi, k_hi - 1);
            for (int i = 0; i < i_end; ++i) {
                const long long jmin = std::max(j_lo, i + 1), jmax = std::min(j_hi, k_hi - 1);
                const long long pmin = jmin * (jmin - 1) / 2 + i, pmax = jmax * (jmax - 1) / 2 + i;
                if (pmin >= pe || pmax < pb) continue;
                t.push_back(make_int4(i, jb, kb, cohort));
            }
        }
    }
}

// The tiles of a whole scan (every pair) in append_tiles order, built on the device from one
// {kb, jb, count, offset} entry per pair of SNP blocks: with every pair in range, each
// i < min(j_hi, k_hi - 1) of a block pair is a tile.
int whole_scan_tiles(epi3_handle* h) {
    const int M = h->M;
    const int kbc = (M + 63) / 64, jbc = (M + 31) / 32;
    std::vector<int4> blocks;
    long long off = 0;
    for (int kb = 0; kb < kbc; ++kb) {
        const int k_hi = std::min(64 * kb + 63, M - 1);
        for (int jb = 0; jb < jbc; ++jb) {
            const int j_lo = 32 * jb, j_hi = std::min(32 * jb + 31, M - 1);
            if (j_lo >= k_hi) continue;
            const int cnt = std::min(j_hi, k_hi - 1);
            if (cnt <= 0) continue;
            blocks.push_back(make_int4(kb, jb, cnt, (int)off));
            off += cnt;
        }
    }
    h->n_tiles = off;
    CK(dev_alloc((void**)&h->d_tiles, sizeof(int4) * (off ? off : 1)), "alloc tiles");
    int4* d_blocks = nullptr;
    CK(dev_alloc((void**)&d_blocks, sizeof(int4) * (blocks.empty() ? 1 : blocks.size())),
       "alloc tile blocks");
    cudaError_t e = cudaSuccess;
    if (!blocks.empty()) {
        e = cudaMemcpyAsync(d_blocks, blocks.data(), sizeof(int4) * blocks.size(),
                            cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_tile_list(d_blocks, (int)blocks.size(), 0, h->d_tiles, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(d_blocks);
    CK(e, "tile list");
    return EPI3_OK;
}

int ensure_tiles(epi3_handle* h, long long pb, long long pe) {
    if (h->d_tiles && h->tiles_pb == pb && h->tiles_pe == pe) return EPI3_OK;
    dev_free(h->d_tiles);
    h->d_tiles = nullptr;
    // whole scan: every pair with a third SNP after it (scan_impl clamps the range to these)
    // (offsets fit int: the tile list is capped)
    if (pb == 0 && pe >= pairs(h->M - 1)) {
        const int rc = whole_scan_tiles(h);
        if (rc != EPI3_OK) return rc;
        h->tiles_pb = pb;
        h->tiles_pe = pe;
        return EPI3_OK;
    }
    std::vector<int4> t;
    append_tiles(h->M, pb, pe, 0, t);
    h->n_tiles = (long long)t.size();
    CK(dev_alloc((void**)&h->d_tiles, sizeof(int4) * (t.empty() ? 1 : t.size())), "alloc tiles");
    if (!t.empty())
        CK(cudaMemcpyAsync(h->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice,
                           h->stream), "upload tiles");
    CK(cudaStreamSynchronize(h->stream), "tiles");
    h->tiles_pb = pb;
    h->tiles_pe = pe;
    return EPI3_OK;
}

// Tiles of the tensor-core form for M SNPs (about M^3 / 12288); the host tile list caps it.
long long mma_tile_estimate(long long M) { return M * M * M / 12288 + 1; }
constexpr long long kMaxMmaTiles = 1LL << 26;

// auto: the path the tuner measured fastest for this shape (tune_handle); with option
// "autotune" = 0, the sample-compacted tensor form, which serves every shape.
int resolve_path(const epi3_handle* h) {
    if (h->path != EPI3_PATH_AUTO) return h->path;
    return h->tuned_path ? h->tuned_path : EPI3_PATH_MMA4C;
}
int tune_handle(epi3_handle* h);

// Candidate stage + result read-back shared by both scan forms.  Returns 1 to retry with a
// larger candidate list, EPI3_OK, or an error.
int finish_scan(epi3_handle* h, int top_k, int attempt) {
    CK(launch_select(h->d_ctrl, h->d_cand, h->cand_cap, top_k, h->k2.rel, h->k2.abs_, h->stream),
       "select launch");
    CK(launch_rescore(h->pl, h->k2, h->d_ctrl, h->d_cand, h->cand_cap, h->d_fin, h->sm_count * 8,
                      h->stream), "rescore launch");
    CK(launch_final(h->d_ctrl, h->d_fin, top_k, h->d_out_scores, h->d_out_trip, h->stream),
       "final launch");
    CK(cudaEventRecord(h->ev[3], h->stream), "event");
    CK(cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream),
       "read status");
    if (!(h->flags & EPI3_DEVICE_PTRS)) {
        CK(cudaMemcpyAsync(h->h_scores, h->d_out_scores, sizeof(double) * top_k,
                           cudaMemcpyDeviceToHost, h->stream), "read scores");
        CK(cudaMemcpyAsync(h->h_trip, h->d_out_trip, sizeof(int) * 3 * top_k,
                           cudaMemcpyDeviceToHost, h->stream), "read triplets");
    }
    CK(cudaStreamSynchronize(h->stream), "scan");
    const int st = h->h_ctrl->status;
    if (st & kStTimeout)
        return fail(EPI3_ERR_TIMEOUT,
                    "a bounded device-side wait of the scan ran out (role %u, tile %u, set %u, step %u, "
                    "detail %#x, %u)", h->h_ctrl->wait_role, h->h_ctrl->wait_tile,
                    h->h_ctrl->wait_set, h->h_ctrl->wait_step, h->h_ctrl->pad_[0], h->h_ctrl->pad_[1]);
    if (st & kStCandOverflow) {
        if (h->cand_cap >= (1LL << 24) || attempt >= 3)
            return fail(EPI3_ERR_OVERFLOW, "more than %lld FP32 candidates", h->cand_cap);
        dev_free(h->d_cand);
        h->d_cand = nullptr;
        h->cand_cap *= 8;
        CK(dev_alloc((void**)&h->d_cand, sizeof(Cand) * h->cand_cap), "grow candidates");
        return 1;
    }
    if (st & kStBadCount)
        return fail(EPI3_ERR_CUDA, "tensor-core tables failed their range check (status %d)", st);
    if (st & kStFinalOverflow)
        return fail(EPI3_ERR_OVERFLOW,
                    "more than %d triplets lie within the FP32 error band of the k-th best",
                    kFinalCap);
    if (st & (kStInternal | kStBadIndex))
        return fail(EPI3_ERR_CUDA, "internal error in the candidate stage (status %d)", st);
    return EPI3_OK;
}

int copy_out(epi3_handle* h, int32_t* out_trip, double* out_scores, int32_t* n_out) {
    const int nout = (int)h->h_ctrl->n_out;
    if (h->flags & EPI3_DEVICE_PTRS) {
        CK(cudaMemcpyAsync(out_scores, h->d_out_scores, sizeof(double) * nout,
                           cudaMemcpyDeviceToDevice, h->stream), "copy scores");
        CK(cudaMemcpyAsync(out_trip, h->d_out_trip, sizeof(int) * 3 * nout,
                           cudaMemcpyDeviceToDevice, h->stream), "copy triplets");
        CK(cudaStreamSynchronize(h->stream), "copy outputs");
    } else {
        memcpy(out_scores, h->h_scores, sizeof(double) * nout);
        memcpy(out_trip, h->h_trip, sizeof(int) * 3 * nout);
    }
    if (n_out) *n_out = nout;
    return EPI3_OK;
}

// Register-split or plain form of the tensor scan for this handle (option "mma_form").
bool mma_split(const epi3_handle* h, int kind) {
    (void)kind;
    return h->mma_form == 0 ? h->tuned_form == 2 : h->mma_form == 2;
}
// Paired epilogue of the compacted form (option "mma_form" = split, or the tuner's choice).
bool cmp_paired(const epi3_handle* h) {
    return h->mma_form == 0 ? (h->tuned_form_path == EPI3_PATH_MMA4C && h->tuned_form == 2)
                            : h->mma_form == 2;
}

CohortDev cohort_of(const epi3_handle* h, long long pb, long long pe, int top_k) {
    CohortDev cd{};
    cd.pl = h->pl;
    cd.k2 = h->k2;
    cd.pt = h->ptab;
    cd.oh = h->d_oh;
    cd.oh_off1 = h->oh_off1;
    {
        const size_t kbc = (size_t)(h->M + 63) / 64, nks = (size_t)h->oh_ks[0] + h->oh_ks[1];
        cd.yoh = h->d_oh ? h->d_oh + kbc * nks * 16384 : nullptr;
        cd.yoh_off1 = (long long)(2 * kbc) * h->oh_ks[0];
        cd.xoh = h->d_oh ? cd.yoh + 2 * kbc * nks * 8192 : nullptr;
        cd.xoh_off1 = (long long)h->M * h->oh_ks[0];
    }
    cd.KS[0] = h->oh_ks[0];
    cd.KS[1] = h->oh_ks[1];
    cd.pair_begin = pb;
    cd.pair_end = pe;
    cd.ctrl = h->d_ctrl;
    cd.cand = h->d_cand;
    cd.cand_cap = h->cand_cap;
    cd.top_k = top_k;
    cd.dbg = h->dbg;
    cd.tsum = h->tsum;
    cd.inject_timeout = inject("timeout") ? 1 : 0;
    return cd;
}

// Operand element kind of a tensor-core path.
int kind_of_path(int path) {
    return path == EPI3_PATH_MMA4 ? kKindE2M1 : (path == EPI3_PATH_MMA ? kKindE4M3 : kKindF16);
}
bool is_mma_path(int path) {
    return path == EPI3_PATH_MMA || path == EPI3_PATH_MMA16 || path == EPI3_PATH_MMA4;
}

int scan_mma_impl(epi3_handle* h, int path, long long pb, long long pe, long long nt, int top_k,
                  int32_t* out_trip, double* out_scores, int32_t* n_out) {
    const int kind = kind_of_path(path);
    if (!h->d_cd) CK(dev_alloc((void**)&h->d_cd, sizeof(CohortDev)), "alloc descriptor");
    const int grid = h->sm_count;
    for (int attempt = 0;; ++attempt) {
        if (inject("launch")) return fail(EPI3_ERR_CUDA, "injected launch failure");
        CK(cudaEventRecord(h->ev[0], h->stream), "event");
        CK(launch_reset(h->d_ctrl, h->stream), "reset launch");
        if (h->tsum)  // a retried scan counts every table again: the checksum restarts with it
            CK(cudaMemsetAsync(h->tsum, 0, 2 * kTsumSlots * sizeof(unsigned long long), h->stream),
               "clear checksum slots");
        CK(cudaEventRecord(h->ev[1], h->stream), "event");
        const CohortDev cd = cohort_of(h, pb, pe, top_k);
        CK(cudaMemcpyAsync(h->d_cd, &cd, sizeof(cd), cudaMemcpyHostToDevice, h->stream),
           "upload descriptor");
        if (h->profile) {
            if (!h->d_prof) CK(dev_alloc((void**)&h->d_prof, 8 * sizeof(unsigned long long)), "alloc profile");
            CK(cudaMemsetAsync(h->d_prof, 0, 8 * sizeof(unsigned long long), h->stream), "clear profile");
        }
        CK(launch_scan_mma(h->d_cd, h->d_tiles, h->n_tiles, kind, grid, h->stream,
                           h->profile ? h->d_prof : nullptr, mma_split(h, kind), h->tsum != nullptr),
           "mma scan launch");
        CK(cudaEventRecord(h->ev[2], h->stream), "event");
        const int rc = finish_scan(h, top_k, attempt);
        if (rc == 1) continue;
        if (rc != EPI3_OK) return rc;
        break;
    }
    const int rc = copy_out(h, out_trip, out_scores, n_out);
    if (rc != EPI3_OK) return rc;
    epi3_stats& s = h->stats;
    s.n_triplets = nt;
    s.n_candidates = h->h_ctrl->n_cand;
    s.n_rescored = h->h_ctrl->n_final;
    s.path = path;
    s.grid = grid;
    s.block = mma_threads(mma_split(h, kind_of_path(path)));
    s.form = mma_split(h, kind_of_path(path)) ? 2 : 1;
    s.kernel_launches = 5;
    s.wait_loader = s.wait_mma_operands = s.wait_mma_accum = s.wait_producers = s.wait_epilogue = 0.f;
    s.wait_producers_tmem = s.mma_issue = 0.f;
    if (h->profile && h->d_prof) {
        unsigned long long p[8];
        CK(cudaMemcpy(p, h->d_prof, sizeof(p), cudaMemcpyDeviceToHost), "read profile");
        const double tot = p[5] > 0 ? (double)p[5] : 1.0;
        s.wait_loader = (float)(p[0] / tot);
        s.wait_mma_operands = (float)(p[1] / tot);
        s.wait_mma_accum = (float)(p[2] / tot);
        s.wait_producers = (float)(p[3] / (tot * 4));
        // the split form's eight epilogue warps each wait; the plain form's one thread waits
        s.wait_epilogue = (float)(p[4] / (tot * (s.block == mma_threads(true) ? 8 : 1)));
        s.wait_producers_tmem = (float)(p[6] / (tot * 4));
        s.mma_issue = (float)(p[7] / tot);
    }
    s.k2_rel_bound = h->k2.rel;
    s.k2_abs_bound = h->k2.abs_;
    s.k2_prune_bound = h->k2.prune_delta;
    s.compact_ms = 0.f;
    cudaEventElapsedTime(&s.scan_kernel_ms, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&s.select_ms, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&s.total_ms, h->ev[0], h->ev[3]);
    (void)cudaGetLastError();
    return EPI3_OK;
}

// Sample-compacted tensor form: the first SNPs are taken in ranges whose compacted chunks fit
// the handle's buffer; per range one compaction launch, then one scan launch over the range's
// tiles (the candidate stage carries over from range to range).

// The compaction plan of the pair range [pb, pe): per first SNP its chunks and tiles, grouped
// into ranges whose chunks fit the handle's buffer; totals of compacted chunks and MMA K-steps
// (the two work terms of this form, used by the tuner to extrapolate a slice's timing).
struct CmpPlan {
    std::vector<CmpFirst> firsts;
    std::vector<int> range_start;   // first SNP of each range
    std::vector<long long> range_chunks, range_tiles;
    size_t need = 0;                // buffer bytes of the largest range
    int i_hi = 0;                   // first SNPs [0, i_hi)
    double chunks_total = 0.0, steps_total = 0.0;
};

void plan_cmp(const epi3_handle* h, long long pb, long long pe, CmpPlan& P) {
    const int M = h->M;
    // pair (i, j) has index j (j - 1) / 2 + i: the pairs of [pb, pe) have j in [j_lo, j_hi];
    // first SNPs i < j_hi, each with the j blocks holding [j_lo, j_hi] (the epilogue drops
    // the pairs outside the range at the ends)
    auto second_of = [](long long p) {
        long long jj = (long long)((1.0 + std::sqrt(1.0 + 8.0 * (double)p)) * 0.5);
        while (jj * (jj - 1) / 2 > p) --jj;
        while ((jj + 1) * jj / 2 <= p) ++jj;
        return jj;
    };
    const long long j_lo = second_of(pb), j_hi = pe > 0 ? second_of(pe - 1) : 0;
    const int i_hi = std::max(0, (int)std::min<long long>(M - 2, j_hi));
    P.i_hi = i_hi;
    const int jb_first = (int)(j_lo / 64), jb_end = (int)(j_hi / 64) + 1;
    std::vector<CmpFirst>& firsts = P.firsts;
    std::vector<int>& range_start = P.range_start;
    std::vector<long long>& range_chunks = P.range_chunks;
    std::vector<long long>& range_tiles = P.range_tiles;
    firsts.assign((size_t)i_hi, CmpFirst{});
    long long chunks = 0, tiles = 0;
    size_t& need = P.need;
    for (int i = 0; i < i_hi; ++i) {
        CmpFirst& f = firsts[i];
        f.b_lo = std::max((i + 1) / 64, jb_first);
        f.jb_end = jb_end;
        // the two least frequent genotypes of SNP i are counted, the third derived
        int n[2][3];
        for (int c = 0; c < 2; ++c) {
            const int2 mg = h->h_marg[(size_t)c * M + i];
            n[c][0] = mg.x;
            n[c][1] = mg.y;
            n[c][2] = (c ? h->N1 : h->N0) - mg.x - mg.y;
        }
        f.drop = cmp_drop(n[0][0] + n[1][0], n[0][1] + n[1][1], n[0][2] + n[1][2]);
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < 2; ++s) f.ks[2 * c + s] = n[c][cmp_geno(f.drop, s)] / 256 + 1;  // + the bias sample
        const long long ch = cmp_chunks_of(f, M);
        if (range_start.empty() || (size_t)(chunks + ch) * 16384 > h->cmp_cap ||
            i - range_start.back() >= 65535) {
            if (!range_start.empty()) {
                range_chunks.push_back(chunks);
                range_tiles.push_back(tiles);
            }
            range_start.push_back(i);
            chunks = 0;
            tiles = 0;
        }
        long long bq = chunks;
        const long long nblk = (M + 63) / 64 - f.b_lo;
        for (int q = 0; q < kCmpSets; ++q) {
            f.base[q] = bq;
            bq += nblk * f.ks[q];
        }
        chunks = bq;
        f.tiles = cmp_tiles_of(M, f.b_lo, f.jb_end);
        f.tile0 = tiles;
        tiles += f.tiles;
        P.chunks_total += (double)(bq - f.base[0]);
        P.steps_total += (double)f.tiles * (f.ks[0] + f.ks[1] + f.ks[2] + f.ks[3]);
        need = std::max(need, (size_t)chunks * 16384);
    }
    if (!range_start.empty()) {
        range_chunks.push_back(chunks);
        range_tiles.push_back(tiles);
    }
}

// The compaction plan of [pb, pe) for this handle, with its first-SNP table uploaded to
// h->d_firsts (the marginals come to the host once per handle).
int cmp_prepare(epi3_handle* h, long long pb, long long pe, CmpPlan& P) {
    const int M = h->M;
    if (h->h_marg.empty()) {
        h->h_marg.resize(2 * (size_t)M);
        CK(cudaMemcpyAsync(h->h_marg.data(), h->d_marg, sizeof(int2) * 2 * (size_t)M,
                           cudaMemcpyDeviceToHost, h->stream), "read marginals");
        CK(cudaStreamSynchronize(h->stream), "read marginals");
    }
    plan_cmp(h, pb, pe, P);
    dev_free(h->d_firsts);
    h->d_firsts = nullptr;
    if (!P.firsts.empty()) {
        CK(dev_alloc((void**)&h->d_firsts, sizeof(CmpFirst) * P.firsts.size()), "alloc first-SNP table");
        CK(cudaMemcpyAsync(h->d_firsts, P.firsts.data(), sizeof(CmpFirst) * P.firsts.size(),
                           cudaMemcpyHostToDevice, h->stream), "upload first-SNP table");
    }
    return EPI3_OK;
}

int scan_cmp_impl(epi3_handle* h, long long pb, long long pe, long long nt, int top_k,
                  int32_t* out_trip, double* out_scores, int32_t* n_out) {
    CmpPlan P;
    const int prc = cmp_prepare(h, pb, pe, P);
    if (prc != EPI3_OK) return prc;
    const std::vector<int>& range_start = P.range_start;
    const std::vector<long long>& range_tiles = P.range_tiles;
    const int i_hi = P.i_hi;
    const size_t need = P.need;
    h->last_cmp_chunks = P.chunks_total;
    h->last_cmp_steps = P.steps_total;
    if (h->cmp_bytes < need) {
        dev_free(h->d_cmp);
        h->d_cmp = nullptr;
        h->cmp_bytes = 0;
        CK(dev_alloc((void**)&h->d_cmp, need), "alloc compacted chunks");
        h->cmp_bytes = need;
    }
    const int grid = h->sm_count;
    const int n_ranges = (int)range_start.size();
    float compact_ms = 0.f;
    while (h->cmp_ev.size() < 2 * (size_t)n_ranges) {  // one event pair per compaction launch
        cudaEvent_t e = nullptr;
        CK(cudaEventCreate(&e), "event create");
        h->cmp_ev.push_back(e);
    }
    for (int attempt = 0;; ++attempt) {
        if (inject("launch")) return fail(EPI3_ERR_CUDA, "injected launch failure");
        CK(cudaEventRecord(h->ev[0], h->stream), "event");
        CK(launch_reset(h->d_ctrl, h->stream), "reset launch");
        if (h->tsum)  // a retried scan counts every table again: the checksum restarts with it
            CK(cudaMemsetAsync(h->tsum, 0, 2 * kTsumSlots * sizeof(unsigned long long), h->stream),
               "clear checksum slots");
        if (h->profile) {
            if (!h->d_prof) CK(dev_alloc((void**)&h->d_prof, 8 * sizeof(unsigned long long)), "alloc profile");
            CK(cudaMemsetAsync(h->d_prof, 0, 8 * sizeof(unsigned long long), h->stream), "clear profile");
        }
        compact_ms = 0.f;
        CK(cudaEventRecord(h->ev[1], h->stream), "event");
        for (int r = 0; r < n_ranges; ++r) {
            const int i0 = range_start[r];
            const int n = (r + 1 < n_ranges ? range_start[r + 1] : i_hi) - i0;
            CK(cudaEventRecord(h->cmp_ev[2 * r], h->stream), "event");
            CK(launch_compact(h->pl, h->d_firsts + i0, i0, n, h->d_cmp, h->stream), "compaction launch");
            CK(cudaEventRecord(h->cmp_ev[2 * r + 1], h->stream), "event");
            CmpArgs a{};
            a.cd = cohort_of(h, pb, pe, top_k);
            a.firsts = h->d_firsts + i0;
            a.i0 = i0;
            a.n_first = n;
            a.n_tiles = range_tiles[r];
            a.cmp = h->d_cmp;
            a.prof = h->profile ? h->d_prof : nullptr;
            CK(launch_scan_cmp(a, grid, h->stream, h->tsum != nullptr || h->profile, cmp_paired(h)),
               "compacted scan launch");
        }
        CK(cudaEventRecord(h->ev[2], h->stream), "event");
        const int rc = finish_scan(h, top_k, attempt);
        if (rc == 1) continue;
        if (rc != EPI3_OK) return rc;
        break;
    }
    for (int r = 0; r < n_ranges; ++r) {  // finish_scan synchronised the stream
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->cmp_ev[2 * r], h->cmp_ev[2 * r + 1]);
        compact_ms += ms;
    }
    const int rc = copy_out(h, out_trip, out_scores, n_out);
    if (rc != EPI3_OK) return rc;
    epi3_stats& s = h->stats;
    s.n_triplets = nt;
    s.n_candidates = h->h_ctrl->n_cand;
    s.n_rescored = h->h_ctrl->n_final;
    s.path = EPI3_PATH_MMA4C;
    s.grid = grid;
    s.block = 512;
    s.form = cmp_paired(h) ? 2 : 1;
    s.kernel_launches = 2 * n_ranges + 3;
    s.wait_loader = s.wait_mma_operands = s.wait_mma_accum = s.wait_producers = s.wait_epilogue = 0.f;
    s.wait_producers_tmem = s.mma_issue = 0.f;
    s.compact_ms = compact_ms;
    h->last_compact_ms = compact_ms;
    if (h->profile && h->d_prof) {
        unsigned long long p[8];
        CK(cudaMemcpy(p, h->d_prof, sizeof(p), cudaMemcpyDeviceToHost), "read profile");
        const double tot = p[5] > 0 ? (double)p[5] : 1.0;
        s.wait_loader = (float)(p[0] / tot);
        s.wait_mma_operands = (float)(p[1] / tot);
        s.wait_mma_accum = (float)(p[2] / tot);
        s.wait_epilogue = (float)(p[4] / tot);
        s.mma_issue = (float)(p[7] / tot);
    }
    s.k2_rel_bound = h->k2.rel;
    s.k2_abs_bound = h->k2.abs_;
    s.k2_prune_bound = h->k2.prune_delta;
    cudaEventElapsedTime(&s.scan_kernel_ms, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&s.select_ms, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&s.total_ms, h->ev[0], h->ev[3]);
    (void)cudaGetLastError();
    return EPI3_OK;
}

int scan_impl(epi3_handle* h, long long pb, long long pe, int top_k, int32_t* out_trip,
              double* out_scores, int32_t* n_out, bool exact_k) {
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    if (!out_trip || !out_scores) return fail(EPI3_ERR_ARG, "null output pointer");
    const long long np = pairs(h->M - 1);  // pairs with j <= M-2 (j = M-1 has no k)
    if (pb < 0 || pe < pb) return fail(EPI3_ERR_ARG, "bad pair range [%lld, %lld)", pb, pe);
    if (pe > np) pe = np;
    if (pb > pe) pb = pe;
    const long long nt = triplets_in_pairs(h->M, pb, pe);
    if (top_k < 1 || top_k > EPI3_MAX_TOPK)
        return fail(EPI3_ERR_ARG, "top_k %d outside 1..%d", top_k, EPI3_MAX_TOPK);
    if (top_k > nt) {
        if (exact_k) return fail(EPI3_ERR_ARG, "top_k %d > %lld triplets", top_k, nt);
        top_k = (int)nt;
    }
    if (n_out) *n_out = 0;
    if (top_k == 0) return EPI3_OK;
    // measure the path (auto) or the tensor-scan form (form auto) once per shape bucket
    if (!h->tuning && h->autotune &&
        ((h->path == EPI3_PATH_AUTO && !h->tuned_path) ||
         ((is_mma_path(resolve_path(h)) || resolve_path(h) == EPI3_PATH_MMA4C) && h->mma_form == 0 &&
          h->tuned_form_path != resolve_path(h)))) {
        const int rc = tune_handle(h);
        if (rc != EPI3_OK) return rc;
    }
    const int path = resolve_path(h);
    if (path != EPI3_PATH_POPC && path != EPI3_PATH_POPC8 && path != EPI3_PATH_MMA4C &&
        !is_mma_path(path))
        return fail(EPI3_ERR_UNSUPPORTED, "path %d not available", path);
    const bool mma = is_mma_path(path);
    if (mma && mma_tile_estimate(h->M) > kMaxMmaTiles)
        return fail(EPI3_ERR_UNSUPPORTED, "n_snps %d too large for the tensor-core tile list", h->M);
    if (path != EPI3_PATH_POPC) {
        int rc = ensure_pair_tables(h);
        if (rc == EPI3_OK && mma) rc = ensure_onehot(h, kind_of_path(path));
        if (rc == EPI3_OK && mma) rc = ensure_tiles(h, pb, pe);
        if (rc != EPI3_OK) return rc;
    }
    if (path == EPI3_PATH_MMA4C) {
        int rc = ensure_pair_tables(h);
        if (rc == EPI3_OK) rc = ensure_pair_floats(h);
        if (rc != EPI3_OK) return rc;
        return scan_cmp_impl(h, pb, pe, nt, top_k, out_trip, out_scores, n_out);
    }
    if (mma) return scan_mma_impl(h, path, pb, pe, nt, top_k, out_trip, out_scores, n_out);

    const int block = h->threads;
    const size_t smem = path == EPI3_PATH_POPC8 ? scan_popc8_smem(h->pl) : scan_popc_smem(h->pl);
    int occ = 0;
    if (path == EPI3_PATH_POPC8) CK(scan_popc8_occupancy(block, smem, &occ), "scan occupancy");
    else CK(scan_popc_occupancy(block, smem, &occ), "scan occupancy");
    if (occ < 1) return fail(EPI3_ERR_UNSUPPORTED, "scan kernel does not fit (smem %zu)", smem);
    const int per_sm = h->ctas_per_sm > 0 && h->ctas_per_sm < occ ? h->ctas_per_sm : occ;
    const int grid = h->sm_count * per_sm;

    for (int attempt = 0;; ++attempt) {
        if (inject("launch")) return fail(EPI3_ERR_CUDA, "injected launch failure");
        CK(cudaEventRecord(h->ev[0], h->stream), "event");
        CK(launch_reset(h->d_ctrl, h->stream), "reset launch");
        if (h->tsum)  // a retried scan counts every table again: the checksum restarts with it
            CK(cudaMemsetAsync(h->tsum, 0, 2 * kTsumSlots * sizeof(unsigned long long), h->stream),
               "clear checksum slots");
        ScanArgs a;
        a.pl = h->pl;
        a.k2 = h->k2;
        a.pt = h->ptab;
        a.ctrl = h->d_ctrl;
        a.cand = h->d_cand;
        a.cand_cap = h->cand_cap;
        a.pair_begin = pb;
        a.pair_end = pe;
        a.top_k = top_k;
        a.dbg = h->dbg;
        a.tsum = h->tsum;
        CK(cudaEventRecord(h->ev[1], h->stream), "event");
        if (path == EPI3_PATH_POPC8) CK(launch_scan_popc8(a, grid, block, smem, h->stream), "scan launch");
        else CK(launch_scan_popc(a, grid, block, smem, h->stream), "scan launch");
        CK(cudaEventRecord(h->ev[2], h->stream), "event");
        CK(launch_select(h->d_ctrl, h->d_cand, h->cand_cap, top_k, h->k2.rel, h->k2.abs_, h->stream),
           "select launch");
        CK(launch_rescore(h->pl, h->k2, h->d_ctrl, h->d_cand, h->cand_cap, h->d_fin,
                          h->sm_count * 8, h->stream),
           "rescore launch");
        CK(launch_final(h->d_ctrl, h->d_fin, top_k, h->d_out_scores, h->d_out_trip, h->stream),
           "final launch");
        CK(cudaEventRecord(h->ev[3], h->stream), "event");
        CK(cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream),
           "read status");
        if (!(h->flags & EPI3_DEVICE_PTRS)) {
            CK(cudaMemcpyAsync(h->h_scores, h->d_out_scores, sizeof(double) * top_k,
                               cudaMemcpyDeviceToHost, h->stream), "read scores");
            CK(cudaMemcpyAsync(h->h_trip, h->d_out_trip, sizeof(int) * 3 * top_k,
                               cudaMemcpyDeviceToHost, h->stream), "read triplets");
        }
        CK(cudaStreamSynchronize(h->stream), "scan");
        const int st = h->h_ctrl->status;
        if (st & kStCandOverflow) {
            if (h->cand_cap >= (1LL << 24) || attempt >= 3)
                return fail(EPI3_ERR_OVERFLOW, "more than %lld FP32 candidates", h->cand_cap);
            dev_free(h->d_cand);
            h->d_cand = nullptr;
            h->cand_cap *= 8;
            CK(dev_alloc((void**)&h->d_cand, sizeof(Cand) * h->cand_cap), "grow candidates");
            continue;
        }
        if (st & kStFinalOverflow)
            return fail(EPI3_ERR_OVERFLOW,
                        "more than %d triplets lie within the FP32 error band of the k-th best",
                        kFinalCap);
        if (st & (kStInternal | kStBadIndex))
            return fail(EPI3_ERR_CUDA, "internal error in the candidate stage (status %d)", st);
        break;
    }
    const int nout = (int)h->h_ctrl->n_out;
    if (h->flags & EPI3_DEVICE_PTRS) {
        CK(cudaMemcpyAsync(out_scores, h->d_out_scores, sizeof(double) * nout,
                           cudaMemcpyDeviceToDevice, h->stream), "copy scores");
        CK(cudaMemcpyAsync(out_trip, h->d_out_trip, sizeof(int) * 3 * nout,
                           cudaMemcpyDeviceToDevice, h->stream), "copy triplets");
        CK(cudaStreamSynchronize(h->stream), "copy outputs");
    } else {
        memcpy(out_scores, h->h_scores, sizeof(double) * nout);
        memcpy(out_trip, h->h_trip, sizeof(int) * 3 * nout);
    }
    if (n_out) *n_out = nout;
    epi3_stats& s = h->stats;
    s.n_triplets = nt;
    s.n_candidates = h->h_ctrl->n_cand;
    s.n_rescored = h->h_ctrl->n_final;
    s.path = path;
    s.grid = grid;
    s.block = block;
    s.kernel_launches = 5;
    s.k2_rel_bound = h->k2.rel;
    s.k2_abs_bound = h->k2.abs_;
    s.k2_prune_bound = h->k2.prune_delta;
    s.form = 0;
    s.compact_ms = 0.f;
    cudaEventElapsedTime(&s.scan_kernel_ms, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&s.select_ms, h->ev[2], h->ev[3]);
    cudaEventElapsedTime(&s.total_ms, h->ev[0], h->ev[3]);
    (void)cudaGetLastError();
    return EPI3_OK;
}

int per_triplet(epi3_handle* h, long long n, const int32_t* trip, int32_t* out_counts,
                float* out_s32, double* out_s64, int path) {
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    if (path == EPI3_PATH_POPC8) {
        const int rc = ensure_pair_tables(h);
        if (rc != EPI3_OK) return rc;
    }
    if (n < 0 || (n > 0 && !trip)) return fail(EPI3_ERR_ARG, "bad triplet list");
    if (n == 0) return EPI3_OK;
    const bool dev = (h->flags & EPI3_DEVICE_PTRS) != 0;
    int* d_trip = nullptr;
    int* d_counts = nullptr;
    float* d_s32 = nullptr;
    double* d_s64 = nullptr;
    int rc = EPI3_OK;
    do {
        cudaError_t e;
        if (dev) {
            d_trip = const_cast<int*>(trip);
            d_counts = out_counts;
            d_s32 = out_s32;
            d_s64 = out_s64;
        } else {
            if ((e = dev_alloc((void**)&d_trip, sizeof(int) * 3 * n)) != cudaSuccess) { rc = cuda_fail(e, "alloc triplets"); break; }
            if ((e = cudaMemcpyAsync(d_trip, trip, sizeof(int) * 3 * n, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "copy triplets"); break; }
            if (out_counts && (e = dev_alloc((void**)&d_counts, sizeof(int) * 54 * n)) != cudaSuccess) { rc = cuda_fail(e, "alloc counts"); break; }
            if (out_s32 && (e = dev_alloc((void**)&d_s32, sizeof(float) * n)) != cudaSuccess) { rc = cuda_fail(e, "alloc s32"); break; }
            if (out_s64 && (e = dev_alloc((void**)&d_s64, sizeof(double) * n)) != cudaSuccess) { rc = cuda_fail(e, "alloc s64"); break; }
        }
        if ((e = launch_reset(h->d_ctrl, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "reset"); break; }
        const bool k2 = out_s32 || out_s64;
        if ((e = launch_tables(h->pl, path == EPI3_PATH_POPC8 ? &h->ptab : nullptr, k2 ? &h->k2 : nullptr, n, d_trip, d_counts, d_s32, d_s64, h->d_ctrl, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "tables launch"); break; }
        if ((e = cudaMemcpyAsync(h->h_ctrl, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read status"); break; }
        if (!dev) {
            if (out_counts && (e = cudaMemcpyAsync(out_counts, d_counts, sizeof(int) * 54 * n, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read counts"); break; }
            if (out_s32 && (e = cudaMemcpyAsync(out_s32, d_s32, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read s32"); break; }
            if (out_s64 && (e = cudaMemcpyAsync(out_s64, d_s64, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess) { rc = cuda_fail(e, "read s64"); break; }
        }
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { rc = cuda_fail(e, "tables"); break; }
        if (h->h_ctrl->status & kStBadIndex) rc = fail(EPI3_ERR_ARG, "triplet index outside 0..%d", h->M - 1);
    } while (0);
    if (!dev) {
        dev_free(d_trip);
        dev_free(d_counts);
        dev_free(d_s32);
        dev_free(d_s64);
    }
    return rc;
}

}  // namespace

void epi3::set_last_error(const char* msg) { g_err = msg; }

extern "C" {

const char* epi3_last_error(void) { return g_err.c_str(); }

int epi3_create(epi3_handle** out, const uint8_t* genotypes, const uint8_t* phenotype,
                int32_t n_snps, int32_t n_samples, int32_t flags, void* cuda_stream) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!out) return fail(EPI3_ERR_ARG, "null handle pointer");
    *out = nullptr;
    if (!genotypes || !phenotype) return fail(EPI3_ERR_ARG, "null genotypes or phenotype");
    if (n_snps < 3) return fail(EPI3_ERR_ARG, "n_snps %d < 3", n_snps);
    if (n_snps >= (1 << 21)) return fail(EPI3_ERR_ARG, "n_snps %d >= 2^21", n_snps);
    if (n_samples < 1) return fail(EPI3_ERR_ARG, "n_samples %d < 1", n_samples);
    if (n_samples > kMaxSamples)
        return fail(EPI3_ERR_UNSUPPORTED, "n_samples %d > %d", n_samples, kMaxSamples);
    if (flags & ~EPI3_DEVICE_PTRS) return fail(EPI3_ERR_ARG, "unknown flags 0x%x", flags);
    int dev = 0, sms = 0;
    int rc = check_device(&dev, &sms);
    if (rc != EPI3_OK) return rc;
    epi3_handle* h = new epi3_handle();
    h->device = dev;
    h->sm_count = sms;
    h->flags = flags;
    h->M = n_snps;
    h->N = n_samples;
    cudaError_t e;
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        release(h);
        return cuda_fail(e, "stream create");
    } else {
        h->own_stream = true;
    }
    for (auto& ev : h->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
            release(h);
            return cuda_fail(e, "event create");
        }
    rc = create_impl(h, genotypes, phenotype);
    if (rc != EPI3_OK) {
        std::string msg = g_err;
        release(h);
        g_err = msg;
        return rc;
    }
    *out = h;
    return EPI3_OK;
}

int epi3_destroy(epi3_handle* h) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    release(h);
    return EPI3_OK;
}

int epi3_scan(epi3_handle* h, int32_t top_k, int32_t* out_triplets, double* out_scores) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    return scan_impl(h, 0, pairs(h->M), top_k, out_triplets, out_scores, nullptr, true);
}

int epi3_scan_range(epi3_handle* h, int64_t pair_begin, int64_t pair_end, int32_t top_k,
                    int32_t* out_triplets, double* out_scores, int32_t* n_out) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    return scan_impl(h, pair_begin, pair_end, top_k, out_triplets, out_scores, n_out, false);
}

int epi3_scan_pairs(epi3_handle* h, int32_t top_k, int32_t* out_pairs, double* out_scores) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    if (!out_pairs || !out_scores) return fail(EPI3_ERR_ARG, "null output pointer");
    const long long np = pairs(h->M);
    if (top_k < 1 || top_k > EPI3_MAX_TOPK || top_k > np)
        return fail(EPI3_ERR_ARG, "top_k %d outside 1..min(%d, %lld)", top_k, EPI3_MAX_TOPK, np);
    int rc = ensure_pair_tables(h);
    if (rc != EPI3_OK) return rc;
    const size_t sel = (pair_scan_scratch(np, top_k) + 255) & ~(size_t)255;
    const size_t need = sel + sizeof(double) * (size_t)top_k + sizeof(int32_t) * 2 * (size_t)top_k;
    if (h->pair_scratch_bytes < need) {
        dev_free(h->d_pair_scratch);
        h->d_pair_scratch = nullptr;
        h->pair_scratch_bytes = 0;
        CK(dev_alloc(&h->d_pair_scratch, need), "alloc pair-scan scratch");
        h->pair_scratch_bytes = need;
    }
    double* d_s = reinterpret_cast<double*>(static_cast<char*>(h->d_pair_scratch) + sel);
    int32_t* d_pairs = reinterpret_cast<int32_t*>(d_s + top_k);
    CK(cudaEventRecord(h->ev[0], h->stream), "event");
    CK(launch_pair_scan(h->ptab, h->k2.lf64, h->M, top_k, h->d_pair_scratch, d_pairs, d_s,
                        h->stream), "pair scan launch");
    CK(cudaEventRecord(h->ev[1], h->stream), "event");
    const cudaMemcpyKind kind =
        (h->flags & EPI3_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(out_pairs, d_pairs, sizeof(int32_t) * 2 * top_k, kind, h->stream),
       "copy pairs");
    CK(cudaMemcpyAsync(out_scores, d_s, sizeof(double) * top_k, kind, h->stream), "copy scores");
    CK(cudaStreamSynchronize(h->stream), "pair scan");
    epi3_stats& s = h->stats;
    s.n_triplets = np;  // pairs scored
    s.n_candidates = 0;
    s.n_rescored = np;
    s.path = EPI3_PATH_AUTO;
    cudaEventElapsedTime(&s.scan_kernel_ms, h->ev[0], h->ev[1]);
    s.total_ms = s.scan_kernel_ms;
    s.select_ms = 0.f;
    (void)cudaGetLastError();
    return EPI3_OK;
}

int epi3_scan_order(epi3_handle* h, int32_t order, int32_t top_k, int32_t* out_snps,
                    double* out_scores) {
    if (order == 2) return epi3_scan_pairs(h, top_k, out_snps, out_scores);
    if (order == 3) return epi3_scan(h, top_k, out_snps, out_scores);
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    if (order < 2 || order > 6)
        return fail(EPI3_ERR_UNSUPPORTED, "interaction order %d (2 to 6 are built)", order);
    if (!out_snps || !out_scores) return fail(EPI3_ERR_ARG, "null output pointer");
    if (h->M < order) return fail(EPI3_ERR_ARG, "order %d needs at least %d SNPs", order, order);
    const long long nq = order_count(h->M, order);
    if (top_k < 1 || top_k > EPI3_MAX_TOPK || top_k > nq)
        return fail(EPI3_ERR_ARG, "top_k %d outside 1..min(%d, %lld)", top_k, EPI3_MAX_TOPK, nq);
    if (h->N0 >= 65536 || h->N1 >= 65536 || h->M >= 65536)
        return fail(EPI3_ERR_UNSUPPORTED, "the %d-SNP scan needs class sizes and n_snps below 65536", order);
    const size_t sel = ((order == 4 ? quad_scan_scratch(h->M, top_k)
                                    : order_scan_scratch(h->M, order, top_k)) + 255) & ~(size_t)255;
    if (sel > (size_t)4 << 30)
        return fail(EPI3_ERR_UNSUPPORTED, "%d-SNP scan of %d SNPs with top_k %d needs %zu bytes of "
                    "selection scratch (limit 4 GiB)", order, h->M, top_k, sel);
    const size_t need = sel + sizeof(double) * (size_t)top_k + sizeof(int32_t) * order * (size_t)top_k;
    if (h->pair_scratch_bytes < need) {
        dev_free(h->d_pair_scratch);
        h->d_pair_scratch = nullptr;
        h->pair_scratch_bytes = 0;
        CK(dev_alloc(&h->d_pair_scratch, need), "alloc k-SNP scan scratch");
        h->pair_scratch_bytes = need;
    }
    double* d_s = reinterpret_cast<double*>(static_cast<char*>(h->d_pair_scratch) + sel);
    int32_t* d_sets = reinterpret_cast<int32_t*>(d_s + top_k);
    CK(cudaEventRecord(h->ev[0], h->stream), "event");
    if (order == 4)
        CK(launch_quad_scan(h->pl, h->k2.lf64, h->N0, h->N1, top_k, h->d_pair_scratch, d_sets, d_s,
                            h->stream), "four-SNP scan launch");
    else
        CK(launch_order_scan(h->pl, h->k2.lf64, order, top_k, h->d_pair_scratch, d_sets, d_s, h->stream),
           "k-SNP scan launch");
    CK(cudaEventRecord(h->ev[1], h->stream), "event");
    const cudaMemcpyKind kind =
        (h->flags & EPI3_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(out_snps, d_sets, sizeof(int32_t) * order * top_k, kind, h->stream),
       "copy sets");
    CK(cudaMemcpyAsync(out_scores, d_s, sizeof(double) * top_k, kind, h->stream), "copy scores");
    CK(cudaStreamSynchronize(h->stream), "k-SNP scan");
    epi3_stats& s = h->stats;
    s.n_triplets = nq;  // sets scored
    s.n_candidates = 0;
    s.n_rescored = nq;
    s.path = EPI3_PATH_POPC;
    cudaEventElapsedTime(&s.scan_kernel_ms, h->ev[0], h->ev[1]);
    s.total_ms = s.scan_kernel_ms;
    s.select_ms = 0.f;
    (void)cudaGetLastError();
    return EPI3_OK;
}

int epi3_tables(epi3_handle* h, int64_t n, const int32_t* triplets, int32_t* out_counts,
                int32_t path) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (path != EPI3_PATH_AUTO && path != EPI3_PATH_POPC && path != EPI3_PATH_POPC8)
        return fail(EPI3_ERR_UNSUPPORTED, "path %d not available", path);
    if (n > 0 && !out_counts) return fail(EPI3_ERR_ARG, "null out_counts");
    return per_triplet(h, n, triplets, out_counts, nullptr, nullptr,
                       path == EPI3_PATH_AUTO ? EPI3_PATH_POPC : path);
}

int epi3_scores(epi3_handle* h, int64_t n, const int32_t* triplets, float* out_k2_f32,
                double* out_k2_f64) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (n > 0 && !out_k2_f32 && !out_k2_f64) return fail(EPI3_ERR_ARG, "no output requested");
    return per_triplet(h, n, triplets, nullptr, out_k2_f32, out_k2_f64, EPI3_PATH_POPC);
}

int epi3_scan_scores(epi3_handle* h, int32_t path, float* out_scores) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h || !out_scores) return fail(EPI3_ERR_ARG, "null argument");
    if (h->M > 512) return fail(EPI3_ERR_ARG, "epi3_scan_scores needs n_snps <= 512");
    const size_t n = (size_t)h->M * h->M * h->M;
    const bool dev = (h->flags & EPI3_DEVICE_PTRS) != 0;
    float* buf = nullptr;
    if (dev) {
        buf = out_scores;
    } else {
        CK(dev_alloc((void**)&buf, n * sizeof(float)), "alloc score cube");
    }
    cudaError_t e = cudaMemsetAsync(buf, 0xFF, n * sizeof(float), h->stream);  // NaN
    const int saved = h->path;
    int rc = e == cudaSuccess ? EPI3_OK : cuda_fail(e, "clear score cube");
    if (rc == EPI3_OK) {
        h->path = path;
        h->dbg = buf;
        int32_t trip[3];
        double sc;
        rc = scan_impl(h, 0, pairs(h->M), 1, trip, &sc, nullptr, true);
        h->dbg = nullptr;
        h->path = saved;
    }
    if (rc == EPI3_OK && !dev) {
        e = cudaMemcpy(out_scores, buf, n * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "read score cube");
    }
    if (!dev) dev_free(buf);
    return rc;
}

int epi3_scan_checksum(epi3_handle* h, int32_t path, uint64_t* out_sum, int64_t* out_count) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h || !out_sum || !out_count) return fail(EPI3_ERR_ARG, "null argument");
    unsigned long long* d = nullptr;
    CK(dev_alloc((void**)&d, 2 * kTsumSlots * sizeof(unsigned long long)), "alloc checksum slots");
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * kTsumSlots * sizeof(unsigned long long), h->stream);
    int rc = e == cudaSuccess ? EPI3_OK : cuda_fail(e, "clear checksum slots");
    const int saved = h->path;
    if (rc == EPI3_OK) {
        h->path = path;
        h->tsum = d;
        int32_t trip[3];
        double sc;
        rc = scan_impl(h, 0, pairs(h->M), 1, trip, &sc, nullptr, true);
        h->tsum = nullptr;
        h->path = saved;
    }
    unsigned long long slots[2 * kTsumSlots];
    if (rc == EPI3_OK) {
        e = cudaMemcpy(slots, d, sizeof(slots), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "read checksum slots");
    }
    dev_free(d);
    if (rc != EPI3_OK) return rc;
    unsigned long long sum = 0, cnt = 0;
    for (int q = 0; q < kTsumSlots; ++q) {
        sum += slots[q];
        cnt += slots[kTsumSlots + q];
    }
    *out_sum = sum;
    *out_count = (int64_t)cnt;
    return EPI3_OK;
}

int epi3_set_option(epi3_handle* h, const char* key, const char* value) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!h || !key || !value) return fail(EPI3_ERR_ARG, "null argument");
    if (!strcmp(key, "path")) {
        if (!strcmp(value, "auto")) h->path = EPI3_PATH_AUTO;
        else if (!strcmp(value, "popc")) h->path = EPI3_PATH_POPC;
        else if (!strcmp(value, "popc8")) h->path = EPI3_PATH_POPC8;
        else if (!strcmp(value, "mma")) h->path = EPI3_PATH_MMA;
        else if (!strcmp(value, "mma16")) h->path = EPI3_PATH_MMA16;
        else if (!strcmp(value, "mma4")) h->path = EPI3_PATH_MMA4;
        else if (!strcmp(value, "mma4c")) h->path = EPI3_PATH_MMA4C;
        else return fail(EPI3_ERR_UNSUPPORTED, "path '%s' not available", value);
        return EPI3_OK;
    }
    if (!strcmp(key, "threads")) {
        const int v = atoi(value);
        if (v < 64 || v > 256 || v % 32) return fail(EPI3_ERR_ARG, "threads %d not in 64..256 step 32", v);
        h->threads = v;
        return EPI3_OK;
    }
    if (!strcmp(key, "ctas_per_sm")) {
        const int v = atoi(value);
        if (v < 0 || v > 32) return fail(EPI3_ERR_ARG, "ctas_per_sm %d not in 0..32", v);
        h->ctas_per_sm = v;
        return EPI3_OK;
    }
    if (!strcmp(key, "profile")) {
        h->profile = atoi(value) != 0;
        return EPI3_OK;
    }
    if (!strcmp(key, "cmp_buffer_mb")) {
        char* end = nullptr;
        const long v = strtol(value, &end, 10);
        if (!end || *end || v < 1 || v > (1L << 20))
            return fail(EPI3_ERR_ARG, "cmp_buffer_mb must be 1..1048576");
        h->cmp_cap = (size_t)v << 20;
        return EPI3_OK;
    }
    if (!strcmp(key, "mma_form")) {
        if (!strcmp(value, "auto")) h->mma_form = 0;
        else if (!strcmp(value, "plain")) h->mma_form = 1;
        else if (!strcmp(value, "split")) h->mma_form = 2;
        else return fail(EPI3_ERR_ARG, "mma_form '%s' not auto, plain or split", value);
        return EPI3_OK;
    }
    if (!strcmp(key, "candidates")) {
        const long long n = atoll(value);
        if (n < 64 || n > (1LL << 28)) return fail(EPI3_ERR_ARG, "candidates %s outside 64..2^28", value);
        dev_free(h->d_cand);
        h->d_cand = nullptr;
        h->cand_cap = n;
        CK(dev_alloc((void**)&h->d_cand, sizeof(Cand) * h->cand_cap), "alloc candidates");
        return EPI3_OK;
    }
    if (!strcmp(key, "autotune")) {
        h->autotune = atoi(value) != 0;
        return EPI3_OK;
    }
    if (!strcmp(key, "timing")) {
        h->timing = atoi(value) != 0;
        return EPI3_OK;
    }
    return fail(EPI3_ERR_ARG, "unknown option '%s'", key);
}

int epi3_get_stats(const epi3_handle* h, epi3_stats* out) {
    if (!h || !out) return fail(EPI3_ERR_ARG, "null argument");
    *out = h->stats;
    return EPI3_OK;
}

int epi3_get_shape(const epi3_handle* h, int32_t* n_snps, int32_t* n_samples,
                   int32_t* n_controls, int32_t* n_cases) {
    if (!h) return fail(EPI3_ERR_ARG, "null handle");
    if (n_snps) *n_snps = h->M;
    if (n_samples) *n_samples = h->N;
    if (n_controls) *n_controls = h->N0;
    if (n_cases) *n_cases = h->N1;
    return EPI3_OK;
}

}  // extern "C"

// ============================================================================ batches
//
// Many independent data sets ("cohorts") of uneven shape scanned together: every cohort is
// packed into its own handle; the cohorts the tuner gives to the tensor-core form share ONE
// persistent tcgen05 launch over the concatenated tile list (tile.w = cohort), the others
// run the 8-cell POPC scan; each cohort then has its own candidate stage.  The whole
// sequence is captured once into a CUDA graph and replayed by every epi3_batch_scan.

struct epi3_batch {
    int n = 0;
    int device = 0, sm_count = 0, flags = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<epi3_handle*> h;
    std::vector<int> path;              // EPI3_PATH_MMA4, EPI3_PATH_MMA4C or EPI3_PATH_POPC8 per cohort
    // compacted-form cohorts: per cohort its ranges of first SNPs (first SNP of each range,
    // tiles of each range, end of the last), all compacting into one shared buffer
    std::vector<std::vector<int>> cmp_start;
    std::vector<std::vector<long long>> cmp_tiles;
    std::vector<int> cmp_end;
    uint8_t* d_cmp = nullptr;
    Ctrl* d_ctrls = nullptr;            // one control block per cohort, contiguous
    Ctrl* h_ctrls = nullptr;            // pinned
    CohortDev* d_cds = nullptr;
    int4* d_tiles = nullptr;
    long long n_tiles = 0;
    bool split = false;                 // register-split form of the tensor scan
    bool form_set = false;              // split measured on the first scan (or forced)
    double* d_scores = nullptr;         // [n][EPI3_MAX_TOPK]
    int* d_trip = nullptr;
    double* h_scores = nullptr;         // pinned
    int* h_trip = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_k = -1;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    epi3_stats stats{};
    float tune_ms = 0.f;
};

namespace {

void batch_release(epi3_batch* b) {
    if (!b) return;
    const bool synced = b->stream && cudaStreamSynchronize(b->stream) == cudaSuccess;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (epi3_handle* h : b->h) {
        if (!h) continue;
        h->d_ctrl = nullptr;  // owned by the batch
        release(h);
    }
    dev_free(b->d_ctrls, synced);
    host_free(b->h_ctrls);
    dev_free(b->d_cds, synced);
    dev_free(b->d_tiles, synced);
    dev_free(b->d_cmp, synced);
    dev_free(b->d_scores, synced);
    dev_free(b->d_trip, synced);
    host_free(b->h_scores);
    host_free(b->h_trip);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// ---------------------------------------------------------------- path tuner
// The faster of the tensor-core and 8-cell POPC forms for a cohort shape, measured: both
// scan kernels are timed on the cohort's heaviest pair slice (pairs with the smallest j,
// about 1/16 of the pairs) and the lower kernel time per triplet wins.  Results are kept
// per (M / 64, N / 1024) bucket for the process, and in the file named by EPI3_TUNE_CACHE
// (lines "device<TAB>SMs<TAB>M/64<TAB>N/1024<TAB>path[<TAB>form<TAB>scope]") across
// processes.  Scope 0 = a batch cohort's path, 1 = a handle's auto path and form, 2 = the
// form of an explicitly chosen tensor path.
struct TuneEntry {
    std::string dev;
    int sms, mb, nb, path;
    int form = 0, scope = 0;
};
std::vector<TuneEntry> g_tune;
bool g_tune_loaded = false;

std::string device_name(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* f = getenv("EPI3_TUNE_CACHE");
    if (!f) return;
    FILE* fp = fopen(f, "r");
    if (!fp) return;
    char line[512];
    while (fgets(line, sizeof(line), fp)) {
        char name[256];
        TuneEntry e;
        const int got = sscanf(line, "%255[^\t]\t%d\t%d\t%d\t%d\t%d\t%d", name, &e.sms, &e.mb,
                               &e.nb, &e.path, &e.form, &e.scope);
        if (got == 5) e.form = e.scope = 0;
        if (got == 5 || got == 7) {
            e.dev = name;
            g_tune.push_back(e);
        }
    }
    fclose(fp);
}

void tune_store(const TuneEntry& e) {
    g_tune.push_back(e);
    const char* f = getenv("EPI3_TUNE_CACHE");
    if (!f) return;
    FILE* fp = fopen(f, "a");
    if (!fp) return;
    fprintf(fp, "%s\t%d\t%d\t%d\t%d\t%d\t%d\n", e.dev.c_str(), e.sms, e.mb, e.nb, e.path, e.form,
            e.scope);
    fclose(fp);
}

// The handle tuner: for path "auto", every scan form that supports the shape -- 8-cell POPC,
// sample-compacted tensor, one-hot tensor in its plain and register-split forms -- is timed
// on the heaviest pair slice (the first pairs, those with the smallest second SNP: at most 1/16
// of the pairs and about 3e13 sample-triplets), after a warm-up on a sixteenth of it, and its
// time is extrapolated to the whole scan by the form's work terms: triplets for the POPC and
// one-hot forms; for the compacted form its compaction (timed apart, scaled by compacted
// chunks) and its MMA K-steps, both from the plan of the whole scan.  The lowest wins.  For an explicitly chosen one-hot tensor path with form "auto", only its two forms
// are timed.  Results are cached per bucket like the batch tuner's.
int tune_handle(epi3_handle* h) {
    const bool want_path = h->path == EPI3_PATH_AUTO;
    const int fixed = want_path ? 0 : h->path;
    struct Choice { int path, form; };
    std::vector<Choice> cands;
    if (want_path) {
        cands.push_back({EPI3_PATH_POPC8, 0});
        cands.push_back({EPI3_PATH_MMA4C, 1});
        cands.push_back({EPI3_PATH_MMA4C, 2});
        if (mma_tile_estimate(h->M) <= kMaxMmaTiles) {
            cands.push_back({EPI3_PATH_MMA4, 1});
            cands.push_back({EPI3_PATH_MMA4, 2});
        }
    } else {
        cands.push_back({fixed, 1});
        cands.push_back({fixed, 2});
    }
    const int scope = want_path ? 1 : 2;
    tune_load();
    const std::string dev = device_name(h->device);
    const int mb = h->M / 64, nb = h->N / 1024;
    for (const TuneEntry& e : g_tune)
        if (e.dev == dev && e.sms == h->sm_count && e.mb == mb && e.nb == nb && e.scope == scope &&
            (scope == 1 || e.path == fixed)) {
            if (want_path) h->tuned_path = e.path;
            h->tuned_form = e.form ? e.form : 1;
            h->tuned_form_path = e.path;
            return EPI3_OK;
        }
    const long long np = pairs(h->M - 1);
    long long pe = std::max(1LL, np / 16);
    while (pe > 1 && (double)triplets_in_pairs(h->M, 0, pe) * h->N > 3e13) pe /= 2;
    const long long pw = std::max(1LL, pe / 16);
    const double nt_full = (double)triplets_in_pairs(h->M, 0, np);
    const double nt_slice = std::max(1.0, (double)triplets_in_pairs(h->M, 0, pe));
    // the tuning scans run plain: no checksum slots, no profile counters
    const int save_path = h->path, save_form = h->mma_form;
    unsigned long long* const save_tsum = h->tsum;
    const bool save_prof = h->profile;
    h->tsum = nullptr;
    h->profile = false;
    h->tuning = true;
    int32_t trip[3 * 10];   // top-10, the usual request: a list sized like a real scan's
    double sc[10];
    int32_t nout = 0;
    int best = -1, rc = EPI3_OK;
    float best_ms = 0.f;
    for (size_t q = 0; q < cands.size() && rc == EPI3_OK; ++q) {
        h->path = cands[q].path;
        h->mma_form = cands[q].form;
        int r = scan_impl(h, 0, pw, 10, trip, sc, &nout, false);
        if (r == EPI3_OK) r = scan_impl(h, 0, pe, 10, trip, sc, &nout, false);
        if (r == EPI3_ERR_UNSUPPORTED) continue;  // this form does not serve the shape
        if (r != EPI3_OK) {
            rc = r;
            break;
        }
        // the slice's time extrapolated to the whole scan by the form's own work terms
        float ms = h->stats.scan_kernel_ms * (float)(nt_full / nt_slice);
        if (cands[q].path == EPI3_PATH_MMA4C && h->last_cmp_chunks > 0.0 && h->last_cmp_steps > 0.0) {
            CmpPlan full;
            plan_cmp(h, 0, np, full);
            const float t_cmp = std::min(h->last_compact_ms, h->stats.scan_kernel_ms);
            ms = t_cmp * (float)(full.chunks_total / h->last_cmp_chunks) +
                 (h->stats.scan_kernel_ms - t_cmp) * (float)(full.steps_total / h->last_cmp_steps);
        }
        if (best < 0 || ms < best_ms) {
            best = (int)q;
            best_ms = ms;
        }
    }
    h->path = save_path;
    h->mma_form = save_form;
    h->tsum = save_tsum;
    h->profile = save_prof;
    h->tuning = false;
    if (rc != EPI3_OK) return rc;
    if (best < 0) return fail(EPI3_ERR_UNSUPPORTED, "no scan form serves %d SNPs", h->M);
    const Choice c = cands[(size_t)best];
    if (want_path) h->tuned_path = c.path;
    h->tuned_form = c.form ? c.form : 1;
    h->tuned_form_path = c.path;
    TuneEntry e;
    e.dev = dev;
    e.sms = h->sm_count;
    e.mb = mb;
    e.nb = nb;
    e.path = c.path;
    e.form = c.form;
    e.scope = scope;
    tune_store(e);
    return EPI3_OK;
}

int tune_path(epi3_batch* b, epi3_handle* h, int* path_out, float* ms) {
    const char* force = getenv("EPI3_BATCH_PATH");
    if (force && !strcmp(force, "mma")) { *path_out = EPI3_PATH_MMA4; return EPI3_OK; }
    if (force && !strcmp(force, "popc8")) { *path_out = EPI3_PATH_POPC8; return EPI3_OK; }
    if (force && !strcmp(force, "mma4c")) { *path_out = EPI3_PATH_MMA4C; return EPI3_OK; }
    // A cohort whose one-hot tensor tiles cannot fill the GPU on their own is latency-bound when
    // timed alone, yet in the batch its tiles share one persistent launch with every other
    // cohort's (its marginal cost there is its tiles' share of that launch, at the
    // throughput-bound rate, several times the POPC forms').  Timing it alone would be biased
    // against the shared launch, so such cohorts take it; the rest get the handle tuner's
    // measured choice for their shape (8-cell POPC, the compacted form in launches of its own,
    // or the shared one-hot launch).
    if (mma_tile_estimate(h->M) < 64LL * b->sm_count) { *path_out = EPI3_PATH_MMA4; return EPI3_OK; }
    const auto t0 = std::chrono::steady_clock::now();
    h->path = EPI3_PATH_AUTO;
    const int rc = tune_handle(h);
    if (rc != EPI3_OK) return rc;
    *path_out = h->tuned_path;
    *ms += std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return EPI3_OK;
}

int batch_capture(epi3_batch* b, int top_k) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // descriptors of the tensor-core cohorts (candidate lists may have grown)
    std::vector<CohortDev> cds(b->n);
    for (int c = 0; c < b->n; ++c) {
        epi3_handle* h = b->h[c];
        cds[c] = cohort_of(h, 0, pairs(h->M - 1), top_k);
    }
    CK(cudaMemcpyAsync(b->d_cds, cds.data(), sizeof(CohortDev) * b->n, cudaMemcpyHostToDevice,
                       b->stream), "upload descriptors");
    // launch shapes and function attributes are settled before capture
    std::vector<int> grid(b->n, 0);
    std::vector<size_t> smem(b->n, 0);
    for (int c = 0; c < b->n; ++c) {
        if (b->path[c] != EPI3_PATH_POPC8) continue;
        epi3_handle* h = b->h[c];
        int occ = 0;
        smem[c] = scan_popc8_smem(h->pl);
        CK(scan_popc8_occupancy(h->threads, smem[c], &occ), "occupancy");
        if (occ < 1) return fail(EPI3_ERR_UNSUPPORTED, "cohort %d does not fit the POPC scan", c);
        grid[c] = b->sm_count * occ;
    }
    for (int c = 0; c < b->n; ++c)  // the compacted scan's function attributes, outside the capture
        if (b->path[c] == EPI3_PATH_MMA4C) {
            CmpArgs none{};
            CK(launch_scan_cmp(none, b->sm_count, b->stream, false, cmp_paired(b->h[c])),
               "compacted scan set-up");
        }
    CK(cudaStreamSynchronize(b->stream), "descriptors");

    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    cudaError_t err = cudaSuccess;
    const char* where = "";
    int where_c = -1;
    int cur_c = -1;
    const char* cur = "";
    auto ok = [&](cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) {
            err = e;
            where = cur;
            where_c = cur_c;
        }
    };
    cur = "reset";
    for (int c = 0; c < b->n; ++c) {
        cur_c = c;
        ok(launch_reset(b->h[c]->d_ctrl, b->stream));
    }
    cur = "tensor scan";
    cur_c = -1;
    if (b->n_tiles > 0)
        ok(launch_scan_mma(b->d_cds, b->d_tiles, b->n_tiles, kKindE2M1, b->sm_count, b->stream,
                           nullptr, b->split));
    cur = "popc8 scan";
    for (int c = 0; c < b->n; ++c) {
        if (b->path[c] != EPI3_PATH_POPC8) continue;
        cur_c = c;
        epi3_handle* h = b->h[c];
        {
            const cudaError_t stale = cudaGetLastError();
            if (stale != cudaSuccess && err == cudaSuccess) {
                err = stale;
                where = "error pending before the POPC launch";
                where_c = c;
            }
        }
        ScanArgs a{};
        a.pl = h->pl;
        a.k2 = h->k2;
        a.pt = h->ptab;
        a.ctrl = h->d_ctrl;
        a.cand = h->d_cand;
        a.cand_cap = h->cand_cap;
        a.pair_begin = 0;
        a.pair_end = pairs(h->M - 1);
        a.top_k = top_k;
        a.dbg = nullptr;
        a.tsum = nullptr;
        ok(launch_scan_popc8(a, grid[c], h->threads, smem[c], b->stream));
        if (err != cudaSuccess && where_c == c && !strcmp(where, "popc8 scan")) {
            char buf[160];
            snprintf(buf, sizeof(buf), "popc8 scan (grid %d, block %d, smem %zu)", grid[c], h->threads,
                     smem[c]);
            static thread_local std::string detail;
            detail = buf;
            where = detail.c_str();
        }
    }
    cur = "compacted scan";
    for (int c = 0; c < b->n; ++c) {
        if (b->path[c] != EPI3_PATH_MMA4C) continue;
        cur_c = c;
        epi3_handle* h = b->h[c];
        const std::vector<int>& rs = b->cmp_start[c];
        for (size_t r = 0; r < rs.size(); ++r) {
            const int i0 = rs[r];
            const int n = (r + 1 < rs.size() ? rs[r + 1] : b->cmp_end[c]) - i0;
            ok(launch_compact(h->pl, h->d_firsts + i0, i0, n, b->d_cmp, b->stream));
            CmpArgs a{};
            a.cd = cds[c];
            a.firsts = h->d_firsts + i0;
            a.i0 = i0;
            a.n_first = n;
            a.n_tiles = b->cmp_tiles[c][r];
            a.cmp = b->d_cmp;
            a.prof = nullptr;
            ok(launch_scan_cmp(a, b->sm_count, b->stream, false, cmp_paired(h)));
        }
    }
    cur = "candidate stage";
    for (int c = 0; c < b->n; ++c) {
        cur_c = c;
        epi3_handle* h = b->h[c];
        ok(launch_select(h->d_ctrl, h->d_cand, h->cand_cap, top_k, h->k2.rel, h->k2.abs_, b->stream));
        ok(launch_rescore(h->pl, h->k2, h->d_ctrl, h->d_cand, h->cand_cap, h->d_fin,
                          b->sm_count * 8, b->stream));
        ok(launch_final(h->d_ctrl, h->d_fin, top_k, b->d_scores + (size_t)c * EPI3_MAX_TOPK,
                        b->d_trip + (size_t)c * 3 * EPI3_MAX_TOPK, b->stream));
    }
    cur = "read-back";
    cur_c = -1;
    ok(cudaMemcpyAsync(b->h_ctrls, b->d_ctrls, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToHost, b->stream));
    ok(cudaMemcpyAsync(b->h_scores, b->d_scores, sizeof(double) * b->n * EPI3_MAX_TOPK,
                       cudaMemcpyDeviceToHost, b->stream));
    ok(cudaMemcpyAsync(b->h_trip, b->d_trip, sizeof(int) * 3 * b->n * EPI3_MAX_TOPK,
                       cudaMemcpyDeviceToHost, b->stream));
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return fail(EPI3_ERR_CUDA, "batch capture (%s, cohort %d): %s", where, where_c,
                    cudaGetErrorString(err));
    }
    if (ec != cudaSuccess) return cuda_fail(ec, "end capture");
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_fail(ei, "graph instantiate");
    b->graph_k = top_k;
    return EPI3_OK;
}

// Batch tensor-form choices of this process, keyed by the batch's shape (device, SMs and every
// cohort's M, N and path), so that re-creating the same batch does not measure again.
std::vector<std::pair<std::string, bool>> g_batch_forms;
std::string batch_signature(const epi3_batch* b) {
    std::string s = device_name(b->device) + "/" + std::to_string(b->sm_count);
    for (int c = 0; c < b->n; ++c)
        s += "/" + std::to_string(b->h[c]->M) + "x" + std::to_string(b->h[c]->N) + "p" +
             std::to_string(b->path[c]);
    return s;
}

}  // namespace

extern "C" {

int epi3_batch_create(epi3_batch** out, int32_t n_cohorts, const epi3_cohort* cohorts,
                      int32_t flags, void* cuda_stream) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!out) return fail(EPI3_ERR_ARG, "null batch pointer");
    *out = nullptr;
    if (n_cohorts < 1 || !cohorts) return fail(EPI3_ERR_ARG, "need at least one cohort");
    if (flags & ~EPI3_DEVICE_PTRS) return fail(EPI3_ERR_ARG, "unknown flags 0x%x", flags);
    int dev = 0, sms = 0;
    int rc = check_device(&dev, &sms);
    if (rc != EPI3_OK) return rc;
    epi3_batch* b = new epi3_batch();
    b->n = n_cohorts;
    b->device = dev;
    b->sm_count = sms;
    b->flags = flags;
    cudaError_t e;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_release(b);
        return cuda_fail(e, "stream create");
    } else {
        b->own_stream = true;
    }
    auto bail = [&](int code) {
        std::string msg = g_err;
        batch_release(b);
        g_err = msg;
        return code;
    };
    for (auto& ev : b->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(cuda_fail(e, "event create"));
    if ((e = dev_alloc((void**)&b->d_ctrls, sizeof(Ctrl) * n_cohorts)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc control blocks"));
    if ((e = host_alloc((void**)&b->h_ctrls, sizeof(Ctrl) * n_cohorts)) != cudaSuccess)
        return bail(cuda_fail(e, "pinned control blocks"));
    b->h.assign(n_cohorts, nullptr);
    b->path.assign(n_cohorts, EPI3_PATH_POPC8);
    for (int c = 0; c < n_cohorts; ++c) {
        const epi3_cohort& co = cohorts[c];
        rc = epi3_create(&b->h[c], co.genotypes, co.phenotype, co.n_snps, co.n_samples, flags,
                         b->stream);
        if (rc != EPI3_OK) {
            g_err = "cohort " + std::to_string(c) + ": " + g_err;
            return bail(rc);
        }
        epi3_handle* h = b->h[c];
        dev_free(h->d_ctrl);              // the batch keeps every control block together
        h->d_ctrl = b->d_ctrls + c;
        if ((rc = ensure_pair_tables(h)) != EPI3_OK) return bail(rc);
    }
    std::vector<int4> tiles;
    size_t cmp_need = 0;
    b->cmp_start.assign(n_cohorts, std::vector<int>());
    b->cmp_tiles.assign(n_cohorts, std::vector<long long>());
    b->cmp_end.assign(n_cohorts, 0);
    for (int c = 0; c < n_cohorts; ++c) {
        epi3_handle* h = b->h[c];
        if ((rc = tune_path(b, h, &b->path[c], &b->tune_ms)) != EPI3_OK) return bail(rc);
        if (b->path[c] == EPI3_PATH_MMA4) {
            if ((rc = ensure_onehot(h, kKindE2M1)) != EPI3_OK) return bail(rc);
            append_tiles(h->M, 0, pairs(h->M - 1), c, tiles);
        } else if (b->path[c] == EPI3_PATH_MMA4C) {
            // its own compaction + scan launches in the graph, ranges planned now
            CmpPlan P;
            if ((rc = ensure_pair_floats(h)) != EPI3_OK) return bail(rc);
            if ((rc = cmp_prepare(h, 0, pairs(h->M - 1), P)) != EPI3_OK) return bail(rc);
            b->cmp_start[c] = P.range_start;
            b->cmp_tiles[c] = P.range_tiles;
            b->cmp_end[c] = P.i_hi;
            cmp_need = std::max(cmp_need, P.need);
        }
        h->path = b->path[c];
    }
    if (cmp_need && (e = dev_alloc((void**)&b->d_cmp, cmp_need)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc compacted chunks"));
    b->n_tiles = (long long)tiles.size();
    // the tensor launch's form (plain or register-split) is measured on the first scan, unless
    // EPI3_BATCH_FORM forces one
    const char* form = getenv("EPI3_BATCH_FORM");
    b->split = form && !strcmp(form, "split");
    b->form_set = tiles.empty() || (form && (!strcmp(form, "split") || !strcmp(form, "plain")));
    if ((e = dev_alloc((void**)&b->d_tiles, sizeof(int4) * (tiles.empty() ? 1 : tiles.size()))) != cudaSuccess)
        return bail(cuda_fail(e, "alloc tiles"));
    if (!tiles.empty() &&
        (e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(e, "upload tiles"));
    if ((e = dev_alloc((void**)&b->d_cds, sizeof(CohortDev) * n_cohorts)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc descriptors"));
    const size_t nk = (size_t)n_cohorts * EPI3_MAX_TOPK;
    if ((e = dev_alloc((void**)&b->d_scores, sizeof(double) * nk)) != cudaSuccess ||
        (e = dev_alloc((void**)&b->d_trip, sizeof(int) * 3 * nk)) != cudaSuccess ||
        (e = host_alloc((void**)&b->h_scores, sizeof(double) * nk)) != cudaSuccess ||
        (e = host_alloc((void**)&b->h_trip, sizeof(int) * 3 * nk)) != cudaSuccess)
        return bail(cuda_fail(e, "alloc batch outputs"));
    *out = b;
    return EPI3_OK;
}

int epi3_batch_scan(epi3_batch* b, int32_t top_k, int32_t* out_triplets, double* out_scores) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    if (!b || !out_triplets || !out_scores) return fail(EPI3_ERR_ARG, "null argument");
    if (top_k < 1 || top_k > EPI3_MAX_TOPK)
        return fail(EPI3_ERR_ARG, "top_k %d outside 1..%d", top_k, EPI3_MAX_TOPK);
    for (int c = 0; c < b->n; ++c) {
        const long long m = b->h[c]->M;
        if (top_k > m * (m - 1) * (m - 2) / 6)
            return fail(EPI3_ERR_ARG, "top_k %d exceeds the triplets of cohort %d", top_k, c);
    }
    // a batch of the same shape measured earlier in this process: its form
    const std::string sig = batch_signature(b);
    if (!b->form_set)
        for (const auto& e : g_batch_forms)
            if (e.first == sig) {
                b->split = e.second;
                b->form_set = true;
            }
    if (!b->form_set) {
        // first scan: replay the batch once in each form of the tensor launch (both give the
        // full result) and keep the faster
        b->form_set = true;
        float t[2] = {0.f, 0.f};
        for (int f = 0; f < 2; ++f) {
            b->split = f == 1;
            b->graph_k = -1;  // capture again with this form
            const int rc = epi3_batch_scan(b, top_k, out_triplets, out_scores);
            if (rc != EPI3_OK) return rc;
            cudaEventElapsedTime(&t[f], b->ev[0], b->ev[4]);
        }
        const bool split = t[1] < t[0];
        g_batch_forms.emplace_back(sig, split);
        if (split == b->split) return EPI3_OK;  // the last replay's result stands
        b->split = split;
        b->graph_k = -1;
    }
    for (int attempt = 0;; ++attempt) {
        if (!b->exec || b->graph_k != top_k) {
            const int rc = batch_capture(b, top_k);
            if (rc != EPI3_OK) return rc;
        }
        if (inject("launch")) return fail(EPI3_ERR_CUDA, "injected launch failure");
        CK(cudaEventRecord(b->ev[0], b->stream), "event");
        CK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
        CK(cudaEventRecord(b->ev[4], b->stream), "event");
        CK(cudaStreamSynchronize(b->stream), "batch scan");
        bool grow = false;
        for (int c = 0; c < b->n; ++c) {
            const int st = b->h_ctrls[c].status;
            epi3_handle* h = b->h[c];
            if (st & kStTimeout) return fail(EPI3_ERR_TIMEOUT, "cohort %d: a bounded wait ran out", c);
            if (st & kStBadCount) return fail(EPI3_ERR_CUDA, "cohort %d: table range check failed", c);
            if (st & kStCandOverflow) {
                if (h->cand_cap >= (1LL << 24) || attempt >= 3)
                    return fail(EPI3_ERR_OVERFLOW, "cohort %d: more than %lld FP32 candidates", c,
                                h->cand_cap);
                dev_free(h->d_cand);
                h->d_cand = nullptr;
                h->cand_cap *= 8;
                CK(dev_alloc((void**)&h->d_cand, sizeof(Cand) * h->cand_cap), "grow candidates");
                grow = true;
            }
            if (st & kStFinalOverflow)
                return fail(EPI3_ERR_OVERFLOW, "cohort %d: more than %d near-tied candidates", c,
                            kFinalCap);
            if (st & (kStInternal | kStBadIndex))
                return fail(EPI3_ERR_CUDA, "cohort %d: internal error (status %d)", c, st);
        }
        if (grow) {
            b->graph_k = -1;  // candidate pointers changed: capture again
            continue;
        }
        break;
    }
    const bool dev = (b->flags & EPI3_DEVICE_PTRS) != 0;
    for (int c = 0; c < b->n; ++c) {
        const int nout = (int)b->h_ctrls[c].n_out;
        if (dev) {
            CK(cudaMemcpyAsync(out_scores + (size_t)c * top_k, b->d_scores + (size_t)c * EPI3_MAX_TOPK,
                               sizeof(double) * nout, cudaMemcpyDeviceToDevice, b->stream), "copy scores");
            CK(cudaMemcpyAsync(out_triplets + (size_t)c * 3 * top_k, b->d_trip + (size_t)c * 3 * EPI3_MAX_TOPK,
                               sizeof(int) * 3 * nout, cudaMemcpyDeviceToDevice, b->stream), "copy triplets");
        } else {
            memcpy(out_scores + (size_t)c * top_k, b->h_scores + (size_t)c * EPI3_MAX_TOPK,
                   sizeof(double) * nout);
            memcpy(out_triplets + (size_t)c * 3 * top_k, b->h_trip + (size_t)c * 3 * EPI3_MAX_TOPK,
                   sizeof(int) * 3 * nout);
        }
    }
    if (dev) CK(cudaStreamSynchronize(b->stream), "copy outputs");
    epi3_stats& s = b->stats;
    s = epi3_stats{};
    int n_mma = 0;
    for (int c = 0; c < b->n; ++c) {
        const long long m = b->h[c]->M;
        s.n_triplets += m * (m - 1) * (m - 2) / 6;
        s.n_candidates += b->h_ctrls[c].n_cand;
        s.n_rescored += b->h_ctrls[c].n_final;
        n_mma += b->path[c] == EPI3_PATH_MMA4;
    }
    s.path = n_mma == b->n ? EPI3_PATH_MMA4 : (n_mma == 0 ? EPI3_PATH_POPC8 : EPI3_PATH_AUTO);
    s.grid = b->sm_count;
    s.block = mma_threads(b->split);
    s.kernel_launches = b->n + (b->n_tiles > 0 ? 1 : 0) + (b->n - n_mma) + 3 * b->n;
    // device time of the whole graph replay (scan kernels + candidate stages + read-back);
    // the scan kernels are > 99 % of it
    cudaEventElapsedTime(&s.total_ms, b->ev[0], b->ev[4]);
    (void)cudaGetLastError();
    s.scan_kernel_ms = s.total_ms;
    s.select_ms = 0.f;
    s.pack_ms = b->tune_ms;
    return EPI3_OK;
}

int epi3_batch_destroy(epi3_batch* b) {
    g_err.clear();
    (void)cudaGetLastError();  // do not report an earlier call's error as ours
    batch_release(b);
    return EPI3_OK;
}

int epi3_batch_get_stats(const epi3_batch* b, epi3_stats* out) {
    if (!b || !out) return fail(EPI3_ERR_ARG, "null argument");
    *out = b->stats;
    return EPI3_OK;
}

int epi3_batch_get_paths(const epi3_batch* b, int32_t* out_paths) {
    if (!b || !out_paths) return fail(EPI3_ERR_ARG, "null argument");
    for (int c = 0; c < b->n; ++c) out_paths[c] = b->path[c];
    return EPI3_OK;
}

int epi3_batch_get_forms(const epi3_batch* b, int32_t* out_forms) {
    if (!b || !out_forms) return fail(EPI3_ERR_ARG, "null argument");
    for (int c = 0; c < b->n; ++c)
        out_forms[c] = b->path[c] == EPI3_PATH_MMA4C ? (cmp_paired(b->h[c]) ? 2 : 1)
                       : b->path[c] != EPI3_PATH_MMA4 ? 0 : !b->form_set ? -1 : b->split ? 2 : 1;
    return EPI3_OK;
}

int epi3_scan_batch(int32_t n_cohorts, const epi3_cohort* cohorts, int32_t top_k,
                    int32_t* out_triplets, double* out_scores, int32_t flags, void* cuda_stream) {
    epi3_batch* b = nullptr;
    int rc = epi3_batch_create(&b, n_cohorts, cohorts, flags, cuda_stream);
    if (rc != EPI3_OK) return rc;
    rc = epi3_batch_scan(b, top_k, out_triplets, out_scores);
    const std::string msg = g_err;
    epi3_batch_destroy(b);
    g_err = msg;
    return rc;
}

}  // extern "C"
