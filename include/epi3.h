/*
 * epi3 -- exhaustive three-way epistasis scan on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library.  The method is the one of arXiv 2201.10956
 * ("Unlocking Personalized Healthcare on Modern CPUs/GPUs: Three-way Gene
 * Interaction Study"):
 *
 *   - Sec. III: a case-control data set of M SNPs x N samples.  Genotype
 *     values are 0 (homozygous major), 1 (heterozygous), 2 (homozygous minor);
 *     the phenotype is 0 (control) or 1 (case).
 *   - Sec. III / Fig. 1: for a SNP triplet (X, Y, Z) the frequency table holds,
 *     for each genotype combination (gX, gY, gZ) in {0,1,2}^3 and each class,
 *     the number of samples showing it.  Here: table[c][cell], c = 0 controls,
 *     c = 1 cases, cell = 9 gX + 3 gY + gZ, X < Y < Z the SNP indices.
 *   - Eq. 1: the Bayesian K2 score of a table, natural log:
 *       K2 = sum_cells [ log((r+1)!) - log(r0!) - log(r1!) ],  r = r0 + r1.
 *   - Sec. III: the solution is the triplet of lowest K2.  The library returns
 *     the top_k lowest under the total order (K2, i, j, k) ascending, so exact
 *     ties are broken by the SNP indices.
 *
 * Every function returns EPI3_OK (0) or a negative EPI3_ERR_* code, and sets a
 * thread-local message readable with epi3_last_error().  Nothing falls back to
 * the CPU: without a usable sm_103 device calls fail with EPI3_ERR_UNSUPPORTED.
 */
#ifndef EPI3_H
#define EPI3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPI3_VERSION 1

/* status codes */
#define EPI3_OK 0
#define EPI3_ERR_ARG (-1)         /* bad pointer, size, genotype > 2, phenotype > 1, top_k */
#define EPI3_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define EPI3_ERR_OOM (-3)         /* device or pinned host allocation failed */
#define EPI3_ERR_TIMEOUT (-4)     /* a bounded device-side wait ran out (about 1 s) */
#define EPI3_ERR_UNSUPPORTED (-5) /* no sm_103 device, or a path/size this build lacks */
#define EPI3_ERR_OVERFLOW (-6)    /* more near-tied candidates than the candidate stage holds */

/* epi3_create flags */
#define EPI3_DEVICE_PTRS 1 /* genotypes/phenotype (and scan outputs) are device pointers */

/* counting paths (epi3_tables, option "path") */
#define EPI3_PATH_AUTO 0
#define EPI3_PATH_POPC 1  /* 27-cell LOP3 AND + POPC over bit planes (Alg. 2 counting) */
#define EPI3_PATH_POPC8 2 /* 8 cells (genotypes 0/1) by AND + POPC, 19 derived exactly from
                             pair tables and marginals */
#define EPI3_PATH_MMA 3   /* tensor cores: the 8 cells as a GEMM of one-hot 0/1 E4M3 operands
                             (tcgen05 kind::f8f6f4, FP32 accumulation), 19 derived */
#define EPI3_PATH_MMA16 4 /* the same GEMM with FP16 operands (tcgen05 kind::f16) */
#define EPI3_PATH_MMA4 5  /* the same GEMM with FP4 E2M1 operands, two per byte, every 32-element
                             block scaled by 2^0 (tcgen05 kind::mxf4, FP32 accumulation); its
                             tile list serves up to 9377 SNPs (EPI3_ERR_UNSUPPORTED beyond) */
#define EPI3_PATH_MMA4C 6 /* 8 cells on sample-compacted FP4 E2M1 operands: per first SNP i, its
                             two least frequent genotypes a are counted (the third is derived
                             with the other 19 cells); per class and counted a the samples with
                             g_i = a are gathered once, and n(a, b, z) = (one-hot rows (j, b)) x
                             (one-hot rows (k, z)) over those samples (tcgen05 kind::mxf4, both
                             operands from shared memory, 4 MACs per counted sample-triplet);
                             any number of SNPs */

#define EPI3_MAX_TOPK 512

typedef struct epi3_handle epi3_handle;

/*
 * Create a handle: split the samples by class, pack genotypes into bit planes
 * on the device (one plane for genotype 0, one for genotype 1, per class; the
 * genotype-2 plane is never stored and is derived by NOR, Sec. IV-A), and
 * build the log-factorial tables of Eq. 1.
 *
 *   genotypes   [n_snps][n_samples] uint8, values 0..2, SNP-major, row stride
 *               n_samples (Sec. III data set D with SNPs as rows).
 *   phenotype   [n_samples] uint8, 0 = control, 1 = case.
 *   n_snps      M >= 3.   n_samples  N >= 1 (at most 131072).
 *   flags       0: genotypes/phenotype are host memory, copied during the call;
 *               EPI3_DEVICE_PTRS: they are device memory on the current device,
 *               read by the pack kernels during the call.
 *   cuda_stream a cudaStream_t the handle issues all its work on, or NULL for a
 *               stream the library creates and owns.
 *
 * The caller keeps ownership of all inputs; the handle keeps only the packed
 * planes.  On error *h is set to NULL.  Values out of range give EPI3_ERR_ARG.
 */
int epi3_create(epi3_handle** h, const uint8_t* genotypes, const uint8_t* phenotype,
                int32_t n_snps, int32_t n_samples, int32_t flags, void* cuda_stream);

/*
 * Exhaustive scan over every triplet i < j < k (Sec. III, Alg. 2): count the
 * 2 x 27 table, score it with K2 (Eq. 1) and keep the top_k lowest.
 *
 *   top_k         1..min(EPI3_MAX_TOPK, C(M,3))  (EPI3_MAX_TOPK = 512).
 *   out_triplets  [top_k][3] int32, (i, j, k) with i < j < k, 0-based.
 *   out_scores    [top_k] double, K2 ascending.
 *
 * Tables are counted exactly (int32).  Every triplet is scored in FP32 from a
 * split log-factorial table; the candidates that can decide the answer (FP32
 * score within the proven FP32 error band of the k-th best) are recounted and
 * rescored in FP64, and the answer is ordered by (FP64 K2, i, j, k).  The
 * returned scores are those FP64 values.  Outputs are host memory unless the
 * handle was created with EPI3_DEVICE_PTRS.  The call returns when the results
 * are written.  EPI3_ERR_OVERFLOW means that more than 8192 triplets tie within
 * the FP32 error band of the k-th best score.
 */
int epi3_scan(epi3_handle* h, int32_t top_k, int32_t* out_triplets, double* out_scores);

/*
 * The scan restricted to the SNP pairs (i, j) whose index in the order
 * (j ascending, then i ascending) lies in [pair_begin, pair_end): all triplets
 * (i, j, k) with k > j of those pairs.  Pair p = j (j - 1) / 2 + i.  Slices
 * that cover [0, C(M,2)) once give, merged by (K2, i, j, k), the full scan's
 * answer, so a scan can be split, resumed or spread over devices.  Outputs as
 * epi3_scan; top_k is clipped to the slice's triplet count and the number of
 * rows written is returned through *n_out.
 */
int epi3_scan_range(epi3_handle* h, int64_t pair_begin, int64_t pair_end, int32_t top_k,
                    int32_t* out_triplets, double* out_scores, int32_t* n_out);

/*
 * Pairwise (second-order) scan: Eq. 1 applied to two SNPs (3^2 cells x {control, case},
 * cell = 3 gX + gY; the paper states the score for any number of interacting SNPs).  Every
 * pair i < j is scored in FP64 from its exact table, summed in cell order 0..8 with the same
 * log-factorial table as the triplet rescoring; the top_k pairs by (K2 ascending, then i, j)
 * are returned.
 *   top_k        1..min(EPI3_MAX_TOPK, C(M,2)).
 *   out_pairs    [top_k][2] int32, i < j, 0-based;  out_scores [top_k] FP64 K2, ascending.
 * Outputs are host memory unless the handle was created with EPI3_DEVICE_PTRS.  Returns
 * EPI3_OK, EPI3_ERR_ARG (bad top_k or null pointers), EPI3_ERR_OOM or EPI3_ERR_CUDA.
 */
int epi3_scan_pairs(epi3_handle* h, int32_t top_k, int32_t* out_pairs, double* out_scores);

/*
 * Scan of any built interaction order (Eq. 1 is stated for any number of interacting SNPs):
 * every set of `order` SNPs x_0 < ... < x_{order-1} gets its 3^order-cell x {control, case}
 * table (cell = the genotypes read as base-3 digits, x_0 most significant: 9 gX + 3 gY + gZ
 * for three) and its K2; the top_k sets by (K2 ascending, then the indices in order) are
 * returned.
 *   order        2 (= epi3_scan_pairs), 3 (= epi3_scan), or 4, 5, 6: every set counted by
 *                AND + POPC over the bit planes (81, 243 or 729 cells, plane 2 by NOR; order 4
 *                one set per thread, orders 5 and 6 one set per warp) and scored in FP64 in
 *                cell order with the rescoring table (needs M >= order, class sizes and M
 *                below 65536, and at most 4 GiB of selection scratch, about
 *                C(M, order) / 2048 * top_k * 32 bytes); other orders give
 *                EPI3_ERR_UNSUPPORTED.
 *   top_k        1..min(EPI3_MAX_TOPK, C(M, order)).
 *   out_snps     [top_k][order] int32, increasing within a row, 0-based.
 *   out_scores   [top_k] FP64 K2, ascending.
 * Outputs are host memory unless the handle was created with EPI3_DEVICE_PTRS.  Errors as
 * epi3_scan_pairs.
 */
int epi3_scan_order(epi3_handle* h, int32_t order, int32_t top_k, int32_t* out_snps,
                    double* out_scores);

/*
 * Release the handle's device memory, stream (if owned) and events.  Device memory of handles
 * and batches goes to a per-process cache instead of back to the driver (the device is
 * synchronised first, as cudaFree would do), and later handles take their buffers from it:
 * creating and destroying a handle per data set then costs no cudaMalloc / cudaFree.  The
 * environment variable EPI3_CACHE_MB (read once) bounds the cache, default 4096 MB per
 * process, oldest blocks released first; 0 turns it off.  An allocation that fails while
 * blocks are cached empties the cache and tries again.
 */
int epi3_destroy(epi3_handle* h);

/* Message of the last failed call on this thread ("" if none). */
const char* epi3_last_error(void);

/*
 * Debug / test: the exact 2 x 27 tables of n listed triplets (Fig. 1).
 *   triplets    [n][3] int32 SNP indices, any three distinct, in the roles
 *               X, Y, Z of the cell index 9 gX + 3 gY + gZ.
 *   out_counts  [n][2][27] int32; row 0 controls, row 1 cases.
 *   path        EPI3_PATH_AUTO (= POPC: direct 27-cell count) or EPI3_PATH_POPC8
 *               (8 cells counted, 19 derived; needs three distinct SNPs).
 * Pointers are host memory unless the handle has EPI3_DEVICE_PTRS.
 */
int epi3_tables(epi3_handle* h, int64_t n, const int32_t* triplets, int32_t* out_counts,
                int32_t path);

/*
 * Debug / test: K2 (Eq. 1) of n listed triplets, both as the scan's FP32 score
 * (out_k2_f32, may be NULL) and as the FP64 rescoring value (out_k2_f64, may be
 * NULL).  Triplets and pointer kinds as epi3_tables.
 */
int epi3_scores(epi3_handle* h, int64_t n, const int32_t* triplets, float* out_k2_f32,
                double* out_k2_f64);

/*
 * Debug / test: the FP32 K2 that the scan kernel of `path` (EPI3_PATH_*) computes for
 * every triplet i < j < k, written to out_scores[(i * M + j) * M + k] (other entries NaN),
 * so the scan kernels' tables can be checked against epi3_scores for every triplet.
 * out_scores holds M^3 floats; n_snps <= 512.  Pointer kind as epi3_tables.
 */
int epi3_scan_scores(epi3_handle* h, int32_t path, float* out_scores);

/*
 * Debug / test: an order-independent checksum of every table that the scan kernel of `path`
 * (EPI3_PATH_*) counts in a full scan of the handle's data set (no pruning), so two counting
 * forms can be compared table by table at any size.  Each triplet i < j < k with class
 * tables r0[27], r1[27] (the controls' and cases' frequency tables of Eq. 1, Sec. III; cell
 * 9 gX + 3 gY + gZ) contributes
 *     f = fold over q = 0..26 of  f * 0x100000001B3 + r0[q] + (r1[q] << 32)   (from f = 0),
 *     hash = mix(f XOR mix((i << 42) | (j << 21) | k)),
 * mix the splitmix64 finaliser (add 0x9E3779B97F4A7C15; xor-shift 30, multiply
 * 0xBF58476D1CE4E5B9; xor-shift 27, multiply 0x94D049BB133111EB; xor-shift 31), all modulo
 * 2^64.  Outputs (host memory): *out_sum = sum of the hashes mod 2^64, *out_count = tables
 * counted (C(M, 3) for a complete scan).  Errors as epi3_scan.
 */
int epi3_scan_checksum(epi3_handle* h, int32_t path, uint64_t* out_sum, int64_t* out_count);

/*
 * Options (strings): "path" = "auto" (the default: the form a tuner measures fastest for the
 * shape, among EPI3_PATH_POPC8, EPI3_PATH_MMA4C and both forms of EPI3_PATH_MMA4 (which serves
 * up to 9377 SNPs); the first auto scan of a (n_snps / 64, n_samples / 1024) bucket
 * times each on the heaviest slice of pairs, at most 1/16 of them, and the choice is kept for
 * the process and appended to the file named by the environment variable EPI3_TUNE_CACHE,
 * if set, for later processes) | "popc" | "popc8" | "mma" | "mma16" | "mma4" | "mma4c";
 * "autotune" = "1" (default) | "0" (no measuring: auto = EPI3_PATH_MMA4C, form plain);
 * "candidates" = initial length of the FP32 candidate list (64 .. 2^28; default 2^20 from
 * 2^22 triplets on, else 2^16; a scan that overflows it grows it 8x and runs again);
 * "threads" = threads per block of the POPC scan kernels (64..256, multiple of 32);
 * "ctas_per_sm" = persistent CTAs per SM of the POPC scans (0 = occupancy maximum);
 * "timing" = "0" | "1" (record CUDA events around the scan's kernels, read back with
 * epi3_get_stats); "profile" = "0" | "1" (per-role wait accounting inside the tensor-core
 * scan kernel, reported in epi3_stats); "mma_form" = "auto" | "plain" | "split" (the
 * tensor-core scan kernel's form: for EPI3_PATH_MMA4 (and mma, mma16) 14 warps with 128
 * registers each, or 16 warps that move registers to the epilogue; for EPI3_PATH_MMA4C an
 * epilogue that takes a lane's triplets one at a time, or both together in f32x2 instructions;
 * "auto" lets the tuner time both for the shape).  Unknown keys or values: EPI3_ERR_ARG, or EPI3_ERR_UNSUPPORTED
 * for a path that is not available.  "cmp_buffer_mb" = device memory (MiB, default 2048) for
 * the compacted chunks of EPI3_PATH_MMA4C: the first SNPs are compacted and scanned in ranges
 * whose chunks fit it (a range needs at least one first SNP's chunks).
 */
int epi3_set_option(epi3_handle* h, const char* key, const char* value);

/* Figures of the last scan of this handle. */
typedef struct {
    int64_t n_triplets;      /* triplets scored */
    int64_t n_candidates;    /* FP32 candidates that reached the global stage */
    int64_t n_rescored;      /* candidates recounted and rescored in FP64 */
    float scan_kernel_ms;    /* counting + FP32 scoring kernel (timing = 1) */
    float select_ms;         /* threshold selection + FP64 rescoring + final sort */
    float total_ms;          /* whole scan, device time (timing = 1) */
    float pack_ms;           /* bit-plane packing at create: plane zeroing + pack kernel */
    int32_t path;            /* EPI3_PATH_* used */
    int32_t grid;            /* CTAs launched by the scan kernel */
    int32_t block;           /* threads per CTA */
    int32_t kernel_launches; /* kernels launched by the last scan */
    float k2_rel_bound;      /* proven |FP32 - FP64| bound: rel * K2 + abs */
    float k2_abs_bound;
    /* tensor-core scan with option "profile" = 1: share of the kernel's cycles each role
       spent waiting (operand loader on free shared-memory stages, MMA issuer on full stages,
       MMA issuer on free accumulators, producer warps on loaded stages, epilogue warps on
       full accumulators, producer warps on free tensor-memory stages) and the share the MMA
       issuer spent issuing tcgen05.mma / commit instructions */
    float wait_loader, wait_mma_operands, wait_mma_accum, wait_producers, wait_epilogue;
    float wait_producers_tmem, mma_issue;
    /* tensor-core scan: a table whose approximate K2 (Stirling's form with the hardware log,
       no table lookups) exceeds the candidate threshold by more than this proven bound is
       skipped without its exact FP32 score; the bound comes from the approximation's error
       measured on the device for every count 0..N+1 */
    float k2_prune_bound;
    /* sample-compacted form (EPI3_PATH_MMA4C): device time of the compaction kernels, a part
       of scan_kernel_ms (0 for the other forms) */
    float compact_ms;
    /* form of the tensor scan that ran: 1 = plain (one-hot: 14 warps of 128 registers;
       compacted: one triplet per lane at a time), 2 = split / paired (one-hot: registers moved
       to the epilogue; compacted: a lane's two triplets in f32x2 instructions); 0 = POPC */
    int32_t form;
} epi3_stats;

int epi3_get_stats(const epi3_handle* h, epi3_stats* out);

/*
 * The whole scan (epi3_create + epi3_scan + epi3_destroy) without allocating memory.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- hosts with a fixed memory budget, or frameworks whose own caching
 * allocator owns the device memory (a raw cudaMalloc/cudaFree there may fail or
 * implicitly synchronise the device).
 *
 *   genotypes, phenotype   device pointers, same layout and values as epi3_create
 *                          (a genotype > 2 or phenotype > 1 gives EPI3_ERR_ARG).
 *   n_snps, n_samples      M >= 3, 1 <= N <= 65536, and the packed planes, tables and
 *                          candidate lists must fit EPI3_NOALLOC_SCRATCH_BYTES (8 MiB:
 *                          about M * N <= 2.5e7, e.g. 1024 x 20000); larger sizes are
 *                          rejected with EPI3_ERR_ARG before any work is issued.
 *   top_k, out_triplets, out_scores   as epi3_scan, but the outputs are device pointers.
 *   cuda_stream            stream to run on (NULL = the legacy default stream).
 *
 * It counts with the 27-cell POPC scan (EPI3_PATH_POPC, about 5 T sample-triplets/s on
 * GB300), not the tensor-core form epi3_scan uses by default, and its candidate list has a
 * fixed 65536 entries with no retry: a data set with more near-tied FP32 candidates gives
 * EPI3_ERR_OVERFLOW where epi3_scan would grow the list.  The answer is the one epi3_scan
 * gives.
 *
 * All scratch lives in one file-scope __device__ array of EPI3_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device current.
 * Calls share the array and it keeps the last call's contents; each call re-initialises
 * what it reads.  Calls are serialised on the host; each reads status words back and
 * synchronises the stream, so the call cannot be recorded into a CUDA graph (do not call it
 * on a capturing stream) and returns when the results are written.  Calls that overlap on
 * the GPU (e.g. from several processes sharing one context) would race on the array.
 */
#define EPI3_NOALLOC_SCRATCH_BYTES (8u << 20)
int epi3_scan_noalloc(const uint8_t* genotypes, const uint8_t* phenotype, int32_t n_snps,
                      int32_t n_samples, int32_t top_k, int32_t* out_triplets,
                      double* out_scores, void* cuda_stream);

/*
 * Batches: many independent data sets ("cohorts") of uneven size scanned together.  Each
 * cohort is packed like epi3_create; a cohort too small to fill the GPU alone joins the
 * shared one-hot tensor launch, every other one gets the handle tuner's measured choice for its
 * shape (8-cell POPC, the compacted tensor form in launches of its own, or the shared one-hot
 * launch; per M/64, N/1024 bucket; persisted in the file named by EPI3_TUNE_CACHE;
 * EPI3_BATCH_PATH = mma | mma4c | popc8 forces one).  The one-hot tensor cohorts share ONE
 * persistent tcgen05 launch over all their tiles; the whole scan + candidate stages + read-back is captured once in a CUDA graph and
 * replayed by every epi3_batch_scan.  The answer of each cohort is the one epi3_scan gives.
 *
 *   cohorts[c]    {genotypes, phenotype, n_snps, n_samples} as epi3_create.
 *   flags         0 or EPI3_DEVICE_PTRS (inputs and outputs are device memory).
 *   out_triplets  [n_cohorts][top_k][3];  out_scores [n_cohorts][top_k].
 *   top_k         1..min(EPI3_MAX_TOPK, C(M,3) of every cohort).
 */
typedef struct {
    const uint8_t* genotypes;
    const uint8_t* phenotype;
    int32_t n_snps;
    int32_t n_samples;
} epi3_cohort;

typedef struct epi3_batch epi3_batch;

int epi3_batch_create(epi3_batch** b, int32_t n_cohorts, const epi3_cohort* cohorts,
                      int32_t flags, void* cuda_stream);
int epi3_batch_scan(epi3_batch* b, int32_t top_k, int32_t* out_triplets, double* out_scores);
int epi3_batch_destroy(epi3_batch* b);
/* Figures of the last epi3_batch_scan: scan_kernel_ms = total_ms = device time of the graph
 * replay; pack_ms holds the tuner's time at create. */
int epi3_batch_get_stats(const epi3_batch* b, epi3_stats* out);
/* The path the tuner chose for each cohort: EPI3_PATH_MMA4 (the shared one-hot tensor launch),
 * EPI3_PATH_MMA4C (compaction + compacted scan launches of its own in the graph) or
 * EPI3_PATH_POPC8.  The environment variable EPI3_BATCH_PATH = "mma" | "mma4c" | "popc8" forces
 * one for every cohort. */
int epi3_batch_get_paths(const epi3_batch* b, int32_t* out_paths);
/* The tensor-scan form of each cohort: 0 = not a tensor cohort, 1 = plain, 2 = register-split
 * (one-hot) or paired (compacted), -1 = not measured yet.  Compacted cohorts take the handle
 * tuner's form for their shape.  All one-hot cohorts share one persistent launch and so one form,
 * measured on the first epi3_batch_scan by replaying the batch in both forms (the environment
 * variable EPI3_BATCH_FORM = "plain" | "split" forces one).  The tile (128 rows (j, b) x 256
 * columns (k, z) of the one-hot operands) is the kernel's only one: the tensor-memory budget
 * of the split form's accumulator ring admits no other. */
int epi3_batch_get_forms(const epi3_batch* b, int32_t* out_forms);
/* One-shot: epi3_batch_create + epi3_batch_scan + epi3_batch_destroy. */
int epi3_scan_batch(int32_t n_cohorts, const epi3_cohort* cohorts, int32_t top_k,
                    int32_t* out_triplets, double* out_scores, int32_t flags, void* cuda_stream);

/* Shape of a handle: M, N, controls, cases. */
int epi3_get_shape(const epi3_handle* h, int32_t* n_snps, int32_t* n_samples,
                   int32_t* n_controls, int32_t* n_cases);

#ifdef __cplusplus
}
#endif

#endif /* EPI3_H */
