// epi3_scan_noalloc: the whole scan without allocating any memory.
//
// Some callers cannot call cudaMalloc: real-time or embedded hosts with a fixed memory
// budget, and frameworks whose caching allocator owns the device memory (a raw
// cudaMalloc/cudaFree there can fail or implicitly synchronise the device).  For them this
// entry point runs the class split, the packing, the 27-cell POPC scan (the counting kernel
// of the popc path, about 5 T sample-triplets/s on GB300; not the tensor-core form that
// epi3_scan picks by default), the candidate band, FP64 rescoring and the final order, with
// every piece of scratch memory (class counts, packed bit planes, log-factorial tables,
// control block, candidate lists) in one file-scope device array of kScratchBytes;
// the log-factorial tables are staged in file-scope host arrays.  The caller passes device
// inputs and device outputs.  The candidate list has a fixed 65536 entries and is not
// grown: a data set with more FP32 candidates gets EPI3_ERR_OVERFLOW (epi3_scan would retry
// with a larger list).
//
// The call reads status words back and synchronises its stream twice, so it cannot be
// recorded into a CUDA graph: do not call it on a capturing stream.
//
// The array belongs to the library image: every GPU that loads the library holds its
// kScratchBytes until the process exits.  All calls share it and it keeps the previous
// call's contents; each call clears what must start at zero (the control block) and
// overwrites the rest before reading it.  Calls are serialised by a host mutex and return
// only when their results are written; calls that overlapped on the GPU (e.g. from two
// processes' streams sharing one context) would race on the array.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "epi3_internal.cuh"

namespace {

using namespace epi3;

constexpr size_t kScratchBytes = EPI3_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxSamples = 65536;
constexpr long long kNoAllocCandCap = 65536;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host staging of the log-factorial tables (no heap allocation).
double h_lf64[kNoAllocMaxSamples + 2];
float2 h_lf2[kNoAllocMaxSamples + 2];

std::mutex g_mu;
void* g_dev_scratch[kMaxDevices] = {};

int err(int code, const char* msg, cudaError_t e = cudaSuccess) {
    char buf[320];
    if (e != cudaSuccess) snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof(buf), "%s", msg);
    set_last_error(buf);
    return code;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t ctrl, counts, planes, lf2, lf64, cand, fin, total;
};

// Offsets inside the scratch array; the planes are sized for the worst class split.
Layout layout(long long M, long long N) {
    Layout L{};
    size_t o = 0;
    L.ctrl = o;   o += up256(sizeof(Ctrl));
    L.counts = o; o += up256(class_counts_len((int)N) * sizeof(int));
    const long long groups = (N + kSamplesPerGroup - 1) / kSamplesPerGroup + 1;
    L.planes = o; o += up256((size_t)2 * groups * M * sizeof(uint4));
    L.lf2 = o;    o += up256((size_t)(N + 2) * sizeof(float2));
    L.lf64 = o;   o += up256((size_t)(N + 2) * sizeof(double));
    L.cand = o;   o += up256((size_t)kNoAllocCandCap * sizeof(Cand));
    L.fin = o;    o += up256((size_t)kFinalCap * sizeof(Final));
    L.total = o;
    return L;
}

#define NA_CK(call, what)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return err(EPI3_ERR_CUDA, what, e_); \
    } while (0)

int scan_noalloc(const uint8_t* geno, const uint8_t* pheno, int M, int N, int top_k,
                 int32_t* out_trip, double* out_scores, cudaStream_t st) {
    if (!geno || !pheno || !out_trip || !out_scores) return err(EPI3_ERR_ARG, "null pointer");
    if (M < 3 || M >= (1 << 21)) return err(EPI3_ERR_ARG, "n_snps must be in 3..2^21-1");
    if (N < 1 || N > kNoAllocMaxSamples)
        return err(EPI3_ERR_ARG, "n_samples must be in 1..65536 for the no-alloc scan");
    const long long ntrip = (long long)M * (M - 1) * (M - 2) / 6;
    if (top_k < 1 || top_k > EPI3_MAX_TOPK || top_k > ntrip)
        return err(EPI3_ERR_ARG, "top_k must be in 1..min(512, C(M,3))");
    const Layout L = layout(M, N);
    if (L.total > kScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "no-alloc scan of %d SNPs x %d samples needs %zu bytes of scratch; the static "
                 "array holds %zu (use epi3_create/epi3_scan)", M, N, L.total, kScratchBytes);
        set_last_error(buf);
        return EPI3_ERR_ARG;
    }
    int dev = 0, major = 0, minor = 0, sms = 0;
    NA_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return err(EPI3_ERR_UNSUPPORTED, "device ordinal >= 64");
    NA_CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev), "attribute");
    NA_CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev), "attribute");
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
    if (major != 10 || minor != 3) return err(EPI3_ERR_UNSUPPORTED, "needs an sm_103 device");

    // Set-up, once per device, with that device current: the device address of the array.
    if (!g_dev_scratch[dev]) {
        void* p = nullptr;
        NA_CK(cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress(scratch)");
        g_dev_scratch[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_dev_scratch[dev]);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + L.ctrl);
    int* counts = reinterpret_cast<int*>(base + L.counts);
    uint4* planes = reinterpret_cast<uint4*>(base + L.planes);
    float2* lf2 = reinterpret_cast<float2*>(base + L.lf2);
    double* lf64 = reinterpret_cast<double*>(base + L.lf64);
    Cand* cand = reinterpret_cast<Cand*>(base + L.cand);
    Final* fin = reinterpret_cast<Final*>(base + L.fin);

    // class split
    NA_CK(launch_reset(ctrl, st), "reset launch");
    NA_CK(launch_class_index(pheno, N, counts, ctrl, st), "class_index launch");
    int hc[2] = {0, 0};
    Ctrl hctrl;
    NA_CK(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, st), "read counts");
    NA_CK(cudaMemcpyAsync(&hctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read status");
    NA_CK(cudaStreamSynchronize(st), "class_index");
    if (hctrl.status & kStBadPhenotype) return err(EPI3_ERR_ARG, "phenotype value > 1");

    Planes pl{};
    pl.planes = planes;
    pl.M = M;
    pl.W4[0] = (hc[0] + kSamplesPerGroup - 1) / kSamplesPerGroup;
    pl.W4[1] = (hc[1] + kSamplesPerGroup - 1) / kSamplesPerGroup;
    pl.coff[0] = 0;
    pl.coff[1] = 2LL * pl.W4[0] * M;
    pl.pad[0] = kSamplesPerGroup * pl.W4[0] - hc[0];
    pl.pad[1] = kSamplesPerGroup * pl.W4[1] - hc[1];
    NA_CK(launch_pack(geno, pheno, M, N, counts, hc[0], hc[1], pl, planes, ctrl, st), "pack launch");
    // the pack kernel flags genotype values > 2 in the control block, which the reset before
    // the scan clears: read it now
    NA_CK(cudaMemcpyAsync(&hctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read status");
    NA_CK(cudaStreamSynchronize(st), "pack");
    if (hctrl.status & kStBadGenotype) return err(EPI3_ERR_ARG, "genotype value > 2");

    // log-factorial tables of Eq. 1: the same recurrence and split as epi3_create
    h_lf64[0] = 0.0;
    for (int i = 1; i < N + 2; ++i) h_lf64[i] = h_lf64[i - 1] + std::log((double)i);
    int e2 = 0;
    std::frexp(h_lf64[N + 1], &e2);
    const int g = 23 - e2;
    for (int i = 0; i < N + 2; ++i) {
        const double hi = std::ldexp(std::nearbyint(std::ldexp(h_lf64[i], g)), -g);
        h_lf2[i].x = (float)hi;
        h_lf2[i].y = (float)(h_lf64[i] - hi);
    }
    NA_CK(cudaMemcpyAsync(lf64, h_lf64, sizeof(double) * (N + 2), cudaMemcpyHostToDevice, st),
          "upload lf64");
    NA_CK(cudaMemcpyAsync(lf2, h_lf2, sizeof(float2) * (N + 2), cudaMemcpyHostToDevice, st),
          "upload lf2");
    K2Tables k2{};
    k2.lf2 = lf2;
    k2.lf64 = lf64;
    k2.rel = std::ldexp(1.0f, -23);
    k2.abs_ = std::ldexp(1.0f, -(g + 13));

    // scan, candidate band, FP64 rescoring, final order
    const size_t smem = scan_popc_smem(pl);
    int occ = 0;
    NA_CK(scan_popc_occupancy(128, smem, &occ), "scan occupancy");
    if (occ < 1) return err(EPI3_ERR_UNSUPPORTED, "scan kernel does not fit");
    ScanArgs a{};
    a.pl = pl;
    a.k2 = k2;
    a.ctrl = ctrl;
    a.cand = cand;
    a.cand_cap = kNoAllocCandCap;
    a.pair_begin = 0;
    a.pair_end = (long long)(M - 1) * (M - 2) / 2;
    a.top_k = top_k;
    a.dbg = nullptr;
    NA_CK(launch_reset(ctrl, st), "reset launch");
    NA_CK(launch_scan_popc(a, sms * occ, 128, smem, st), "scan launch");
    NA_CK(launch_select(ctrl, cand, kNoAllocCandCap, top_k, k2.rel, k2.abs_, st), "select launch");
    NA_CK(launch_rescore(pl, k2, ctrl, cand, kNoAllocCandCap, fin, sms * 8, st), "rescore launch");
    NA_CK(launch_final(ctrl, fin, top_k, out_scores, out_trip, st), "final launch");
    NA_CK(cudaMemcpyAsync(&hctrl, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read status");
    NA_CK(cudaStreamSynchronize(st), "scan");
    if (hctrl.status & kStCandOverflow)
        return err(EPI3_ERR_OVERFLOW, "more FP32 candidates than the static candidate list holds");
    if (hctrl.status & kStFinalOverflow)
        return err(EPI3_ERR_OVERFLOW, "more than 8192 triplets lie within the FP32 error band");
    if (hctrl.status & (kStInternal | kStBadIndex))
        return err(EPI3_ERR_CUDA, "internal error in the candidate stage");
    return EPI3_OK;
}

}  // namespace

extern "C" int epi3_scan_noalloc(const uint8_t* genotypes, const uint8_t* phenotype,
                                 int32_t n_snps, int32_t n_samples, int32_t top_k,
                                 int32_t* out_triplets, double* out_scores, void* cuda_stream) {
    std::lock_guard<std::mutex> lock(g_mu);
    set_last_error("");
    return scan_noalloc(genotypes, phenotype, n_snps, n_samples, top_k, out_triplets, out_scores,
                        (cudaStream_t)cuda_stream);
}
