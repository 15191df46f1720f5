/*
 * stark.h -- C ABI of libstark.so: Strassen matrix multiplication C = A*B on
 * one NVIDIA GB300 (sm_103a), after "Stark: Fast and Scalable Strassen's
 * Matrix Multiplication using Apache Spark" (arXiv 1811.07325).
 *
 * The method (Alg. 1, Sec. III-A): split A and B into 2x2 quadrants, form the
 * operand sums of the seven products M1..M7, multiply, and recombine
 * C11 = M1+M4-M5+M7, C12 = M3+M5, C21 = M2+M4, C22 = M1-M2+M3+M6 (the paper
 * prints -M3 in C22; +M3 is the identity that equals A*B).  Recursing `depth`
 * times gives 7^depth leaf products of side L = n_pad / 2^depth.  Stark runs
 * every recursion level at once by tagging blocks with their M-index path
 * (Sec. III-B, Alg. 3-5); here the tags are a device-resident table, the
 * divide phase is one kernel that writes every leaf operand, the leaves are
 * one tensor-core launch, and the combine runs in that launch's epilogue.
 *
 * Conventions (all entry points):
 *  - Matrices are square, row-major, contiguous, leading dimension n.
 *  - "Device pointer" means memory of the current CUDA device; "host pointer"
 *    means ordinary (preferably pinned) host memory.  The caller owns every
 *    pointer it passes; the library never frees caller memory.
 *  - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *    default stream).  Calls taking a stream are asynchronous on it unless
 *    stated otherwise; inputs must stay alive and unmodified until the work
 *    completes on that stream.
 *  - Every call returns a stark_status; no call aborts the process.  CUDA
 *    runtime failures map to STARK_ECUDA, a device-side timeout (a bounded
 *    wait inside a kernel that gave up) to STARK_ETIMEOUT.
 *  - A plan may be used by one stream at a time; different plans are
 *    independent.
 */
#ifndef STARK_H
#define STARK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STARK_API __attribute__((visibility("default")))
#else
#define STARK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  STARK_F64 = 0,            /* fp64 in/out; fp64 leaves on CUDA cores                  */
  STARK_F32_SPLIT_BF16 = 1, /* fp32 in/out; leaves as 3 bf16 products (hi*hi + hi*lo +  */
                            /* lo*hi, x = hi + lo) on tcgen05 tensor cores, fp32 accum. */
  STARK_F32_SPLIT_TF32 = 2, /* fp32 in/out; the same with TF32 halves                   */
  STARK_I64 = 3,            /* int64 in/out; exact modulo 2^64 (two's complement)       */
  STARK_F32_SPLIT_FP16 = 4  /* fp32 in/out; the same with IEEE fp16 halves (11 bits     */
                            /* each: about 22 bits per operand at the bf16 MMA rate).   */
                            /* Every leaf operand sum must stay below 65504 in         */
                            /* magnitude: a larger one sets the plan's device range    */
                            /* flag (stark_plan_check: STARK_EINVAL, product invalid). */
                            /* Sums below 2^-14 keep their fp16 value to 2^-24 (an     */
                            /* absolute error of at most 2^-25 per split).             */
                            /* stark_mul_noalloc is 3xBF16 only.                        */
} stark_dtype;

typedef enum {
  STARK_OK = 0,
  STARK_EINVAL = 1,      /* bad argument (null pointer, n < 0, depth out of range, ...) */
  STARK_ENOMEM = 2,      /* device or host allocation failed, or over the memory budget */
  STARK_EUNSUPPORTED = 3,/* valid request the library or device cannot serve          */
  STARK_ETIMEOUT = 4,    /* a bounded device-side wait expired; results are invalid    */
  STARK_EBUSY = 5,       /* the request is still queued or running                      */
  STARK_ENOTFOUND = 6,   /* unknown request id                                           */
  STARK_ECUDA = 7        /* a CUDA runtime call failed                                   */
} stark_status;

typedef struct stark_plan_s *stark_plan_t;

/* What a plan decided; filled by stark_plan_get_info. */
typedef struct {
  int64_t n;               /* problem side                                              */
  int64_t n_pad;           /* recursion's padded side: multiple of 2^depth * granularity */
  int64_t leaf;            /* L = n_pad / 2^depth                                        */
  int32_t depth;           /* recursion levels                                           */
  int32_t dtype;           /* stark_dtype                                                 */
  int64_t leaves;          /* 7^depth                                                    */
  int64_t workspace_bytes; /* device bytes the plan owns (leaf operands, tables, ...)    */
  int32_t tile_m, tile_n;  /* leaf GEMM output tile                                      */
  int32_t peel;            /* edge rows/columns done classically (STARK_PLAN_PEEL), else 0 */
  int32_t combine;         /* combine mode in effect (stark_plan_set_combine)            */
  int32_t shard_levels;    /* stark_plan_set_shard: top levels above the shard's subtrees (0: none) */
  int32_t shard_first;     /* first leaf whose operands the shard's workspace holds     */
  int32_t workspace_leaves;/* leaves whose operands the workspace holds (all of them, one  */
                           /* depth-first subtree's, or a shard's subtrees')               */
  int32_t promotion_k;     /* stark_plan_set_promotion: K per tensor-core accumulation, 0: off */
} stark_plan_info;

/* ----------------------------------------------------------------- plans */

/* Build a plan for n x n products with `depth` recursion levels (Alg. 1 /
 * Alg. 2: depth = log2 of the number of partitions per side, the paper's
 * p - q).  depth = -1 lets the library choose: for the tensor-core dtypes a
 * measured autotuner times the candidate depths on the device once per size
 * class (n rounded up to 64, 128 or 256) and caches the winner for the process (the
 * paper's U-shaped optimum over the partition count, Sec. V-C, found by
 * measurement); for F64/I64 a cost model over leaf work and divide traffic.
 * depth 0 multiplies classically (one leaf).
 * Allocates the plan's device workspace on the current device.
 * Errors: EINVAL (n < 0 or > 2^20, depth < -1 or > 4, unknown dtype, out == NULL),
 * ENOMEM, ECUDA, EUNSUPPORTED (current device is not a GB300 / sm_103). */
STARK_API stark_status stark_plan(int64_t n, int depth, stark_dtype dtype, stark_plan_t *out);

/* Plan options for stark_plan_ex.
 * STARK_PLAN_PEEL: edge peeling instead of padding for sizes the tiling does
 *   not divide.  With g = 2^depth * 128 (64 for F64/I64), n = m + r and m the
 *   largest multiple of g not above n, the recursion runs on the m x m core
 *   of A and B (no padding) and three classical products on the CUDA cores
 *   finish C: C[:m,:m] += A[:m,m:] B[m:,:m], C[:m,m:] = A[:m,:] B[:,m:],
 *   C[m:,:] = A[m:,:] B (block form of A B; fp32 FMA for the split dtypes,
 *   fp64, or wrapping int64).  Padding costs (n_pad^3 - n^3) extra tensor
 *   work; peeling costs about 6 n^2 r CUDA-core operations, so it pays for
 *   small r (n just above a multiple of g).  No effect when g divides n or
 *   n < g; stark_plan_info.peel reports r. */
#define STARK_PLAN_PEEL 1u

/* stark_plan with options (a bitwise OR of STARK_PLAN_* flags; 0 is
 * stark_plan).  Errors as stark_plan, and EINVAL for unknown flags. */
STARK_API stark_status stark_plan_ex(int64_t n, int depth, stark_dtype dtype, unsigned flags, stark_plan_t *out);

/* Release a plan and its workspace (waits for the device to finish using it).
 * NULL is accepted and ignored. */
STARK_API stark_status stark_plan_destroy(stark_plan_t plan);

STARK_API stark_status stark_plan_get_info(stark_plan_t plan, stark_plan_info *info);

/* C = A * B: Strassen's recursion (Alg. 1, Sec. III-A) run as Stark runs it,
 * every level at once (Alg. 2, Sec. III-C): the divide (Alg. 3) forms every
 * leaf operand sum, the leaf products (Alg. 4) multiply them, and the
 * combine (Alg. 5) adds each product into C with its signs.
 * A, B, C: device pointers to n x n matrices of the plan's
 * element type (double, float, float, int64_t).  C is overwritten; it may not
 * alias A or B.  Enqueues: zero C, divide A, divide B, one leaf-product launch
 * whose epilogue accumulates every leaf into C with the combine signs.
 * Asynchronous on `stream`; capturable in a CUDA graph (no allocation, no
 * synchronisation).  n == 0 is a no-op. */
STARK_API stark_status stark_mul(stark_plan_t plan, const void *A, const void *B, void *C, void *stream);

/* The same product, end to end from host memory: copies A and B host->device
 * into plan-owned buffers, runs stark_mul, copies C device->host and waits
 * for completion (then reports device-side errors like stark_plan_check).
 * A, B, C: host pointers (pinned memory gives full copy bandwidth).
 * Synchronous.  Allocates two staging sets (6 n^2 elements) on first use. */
STARK_API stark_status stark_mul_host(stark_plan_t plan, const void *A, const void *B, void *C, void *stream);

/* Asynchronous form of stark_mul_host for streams of products: enqueues the
 * host->device copies, the product and the device->host copy on three
 * plan-owned streams with alternating staging sets, so the copies of one
 * call overlap the product of the previous one, and makes `stream` wait for
 * this product's result.  The host buffers must stay valid and unmodified
 * (C unread) until `stream` has passed that point.  Copies out run in call
 * order, so a C buffer passed again to a later call ends up holding the
 * later result; read it in between only after the earlier call completed.
 * Errors as stark_mul. */
STARK_API stark_status stark_mul_host_async(stark_plan_t plan, const void *A, const void *B, void *C,
                                            void *stream);

/* The same pipeline without a wait on a caller's stream: enqueues the copy
 * in and the product and returns; the copy out of this product is enqueued
 * by the next call (after that call's copy in), by stark_plan_host_wait or by
 * stark_plan_destroy, and stark_plan_host_wait collects every product
 * enqueued so far.  CUDA multiplexes streams onto a few hardware queues; an
 * operation that waits on a later event holds back everything queued behind
 * it in a shared queue, so this form enqueues operations in the order they
 * become ready and puts no wait on any stream it does not own.  Copies in
 * one direction still wait behind copies in the other when the plan's copy
 * streams share a queue (then each product costs the two copies one after
 * the other, about 17.6 ms at n = 16384 instead of the product's 13.9): a
 * process with many streams should raise CUDA_DEVICE_MAX_CONNECTIONS (read
 * when CUDA starts; 8 by default) to 32 so the plan's streams get queues
 * of their own.  (stark_mul_host_async's wait on `stream` can hold back
 * the next call's copies when `stream` shares a queue with the plan's.)
 * Buffer rules as stark_mul_host_async, with "until stark_plan_host_wait
 * returned" for "until `stream` has passed that point".  Errors as
 * stark_mul. */
STARK_API stark_status stark_mul_host_enqueue(stark_plan_t plan, const void *A, const void *B, void *C);

/* Blocks until every product enqueued with stark_mul_host_enqueue (or
 * stark_mul_host_async) has its C in host memory, then reports the device
 * error word as stark_plan_check does.  OK at once when nothing is pending. */
STARK_API stark_status stark_plan_host_wait(stark_plan_t plan);

/* Partial product for sharding the leaves across devices (the independent
 * products of one recursion tree, Sec. III-C): C = sum over leaves l in
 * [leaf_begin, leaf_end) of that leaf's signed combine contributions.
 * Summing the C of any partition of [0, 7^depth) gives A*B.  Same pointer
 * rules as stark_mul. */
STARK_API stark_status stark_mul_leaves(stark_plan_t plan, const void *A, const void *B, void *C, int64_t leaf_begin,
                              int64_t leaf_end, void *stream);

/* Divide phase only (Alg. 3): writes every leaf operand of A and of B into
 * the plan's workspace and returns read-only device pointers to it, for
 * inspection by tests.  Layout: split dtypes hold [2*leaves][L][L] planes
 * (hi planes, then lo planes; bf16 values, or TF32 values in fp32
 * containers); F64/I64 hold [leaves][L][L].  Every plane is row-major: A
 * planes are the leaf's M x K operand, B planes its K x N operand, except
 * for F32_SPLIT_TF32 with the K-major layout (stark_plan_set_tf32_layout 0),
 * whose B planes are stored transposed (N x K).  A plan restricted by
 * stark_plan_set_shard holds the operands of its subtrees' leaves only
 * (stark_plan_info.workspace_leaves of them, from leaf shard_first on).  The
 * pointers stay valid until the plan is destroyed and are overwritten by the
 * next product. */
STARK_API stark_status stark_plan_operands(stark_plan_t plan, const void *A, const void *B, void *stream, const void **X,
                                 const void **Y);

/* How the combine (Alg. 5) adds leaf tiles into C on the tensor-core dtypes:
 * mode 0 (default) fuses it into the leaf epilogue with TMA bulk
 * add-reductions of 32 x 32 boxes (through an aligned staging copy of C when
 * n is not a multiple of 4); mode 1 fuses it with signed vector atomics;
 * mode 2 is deterministic: the leaf epilogue stores every product M_l
 * (allocating [leaves][L][L] fp32 planes) and a separate pass writes each C
 * element once as its signed sum in ascending leaf order, so results are
 * bitwise reproducible run to run (depth <= 3; stark_mul_leaves keeps the
 * fused path); mode 3 folds the last recursion level on the way: the CTA
 * pairs run the seven children of one parent product back to back at one
 * tile position, and each child's tile is stored (first child of a
 * quadrant) or added (the others) into that quadrant of the parent's
 * product, held in [leaves/7][2L][2L] fp32 planes that stay in L2 while the
 * siblings run; an ordered pass then combines the parent products into C as
 * mode 2 does one level up (C written once; bitwise reproducible).  Mode 3
 * needs depth >= 1, a leaf side that is a multiple of 256, breadth-first
 * traversal and (3xTF32) the MN-major layout; a product it cannot serve
 * (stark_mul_leaves, another pairing or pipeline) runs the fused path.
 * All modes agree within fp32 rounding (the order of the additions
 * differs).  mode -1 measures: every mode that applies to the plan runs one
 * warm-up and three timed products on scratch inputs (allocated for the
 * call), the fastest stays in effect (stark_plan_info.combine) and the
 * product buffers of the others are released; F64/I64 plans keep mode 0.
 * Errors: EINVAL, EUNSUPPORTED (mode 2 on an fp64/int64 plan or depth > 3;
 * mode 3 outside its conditions), ENOMEM, ETIMEOUT (a trial product's
 * device wait expired). */
STARK_API stark_status stark_plan_set_combine(stark_plan_t plan, int mode);

/* Leaf launch schedule of the split-fp32 paths (Alg. 4 leaf products), for leaf
 * sides that allow it (256-wide tiles, L a multiple of 256):
 *   0  single CTAs, each a 128 x 256 tile;
 *   2  CTA pairs sharing one 256 x 256 tensor-core MMA (cta_group::2): each
 *      CTA stages half of the A rows and half of the B columns (3xBF16 and
 *      3xTF32; the default).
 * Other leaf sides run mode 0.  Mode 1 (tiles shared between the CTAs of a
 * cluster by multicast loads) is not offered.  Results agree within fp32
 * rounding of the combine's order.  Errors: EINVAL (null plan, mode outside
 * 0..2), EUNSUPPORTED (mode 1; the plan keeps its schedule). */
STARK_API stark_status stark_plan_set_pairing(stark_plan_t plan, int enable);

/* Order of a leaf's output tiles in the split-fp32 leaf launch: band > 0
 * runs them in bands of `band` tile columns (row-major within a band), so
 * the tiles in flight at one time share fewer B panels; 0 (default) is
 * row-major over the whole leaf.  A band that does not divide the leaf's
 * tile columns means row-major.  Results agree within fp32 rounding of the
 * combine's order.  Errors: EINVAL (null plan, band < 0 or > 4096). */
STARK_API stark_status stark_plan_set_raster(stark_plan_t plan, int band);

/* Layout of the 3xTF32 path's B operand (the leaf planes Y_l): mn = 0
 * transposes the planes in place after the divide and reads them K-major;
 * mn = 1 (default) keeps them row-major (K x N) and reads them MN-major with
 * the 128-byte swizzle of 32-byte atoms, with no transpose pass.  Errors:
 * EINVAL (null plan, mn outside 0..1), EUNSUPPORTED (mn = 1 on a plan of
 * another dtype). */
STARK_API stark_status stark_plan_set_tf32_layout(stark_plan_t plan, int mn);

/* Accumulator promotion for the split-fp32 leaf products (the leaf GEMMs of
 * Alg. 4; the paper's leaves are FP64 and need none).  The tensor core sums
 * a leaf tile's products over K in its fp32 accumulator; its additions do
 * not round to nearest, so their error grows with the number of K steps.
 * k_chunk > 0 limits one tensor-core accumulation to k_chunk of K: after
 * each chunk the partial tile is added to a running fp32 sum on the CUDA
 * cores (round to nearest), and the running sum is what the combine sees.
 * k_chunk = 0 (default) accumulates over the whole leaf side.  The running
 * sum lives in the registers of the kernel's epilogue warps and the two TMEM
 * accumulators alternate between chunks, so the MMAs do not wait for the
 * additions; the cost is the TMEM reads of each chunk (measured at
 * n = 16384, depth 2: 3xTF32 383 -> 382, 3xFP16 677 -> 654 TFLOP/s with
 * k_chunk = 256).  Applies to the CTA-pair leaf kernel:
 * leaf side a multiple of 256, 256-wide tiles, 3xBF16, 3xFP16 or 3xTF32
 * with the MN-major layout, combine modes 0-2.  Errors: EINVAL (null plan, k_chunk
 * < 0 or not a multiple of 256), EUNSUPPORTED (another dtype, leaf side or
 * layout, or combine mode 3; a later product whose leaves would run on
 * another kernel also returns EUNSUPPORTED). */
STARK_API stark_status stark_plan_set_promotion(stark_plan_t plan, int k_chunk);

/* Operand pipeline of the 3xBF16 leaf launch with 256-wide tiles: deep = 1
 * runs single CTAs that stage K = 32 per step in four 48 KB buffers
 * (64-byte swizzle), in place of the leaf schedule of
 * stark_plan_set_pairing; 0 (default) keeps that schedule (CTA pairs: K = 64
 * in three 64 KB buffers per CTA; single CTAs: two 96 KB buffers).  Same
 * results up to the combine's addition order.  Errors: EINVAL. */
STARK_API stark_status stark_plan_set_pipeline(stark_plan_t plan, int deep);

/* Traversal of the recursion tree (memory-lean form; the paper names the
 * O(3^l N^2) space growth as Stark's drawback, Sec. VI).
 * levels = 0 (default): breadth first, one divide for all 7^d leaves and
 * one leaf launch.  levels = k (1, or 2 for the split-fp32 dtypes): depth
 * first over the top k levels: for each of the 7^k products there, divide
 * only its subtree (reading A and B through that product's level-1..k
 * operand sums, formed on the fly in the order of Alg. 1) and launch its
 * 7^(d-k) leaves; the workspace shrinks 7^k-fold (the plan reallocates it),
 * the divide reads A and B 3^k times over.  Results agree within the
 * combine's rounding order (bit-identical for int64).  Errors: EINVAL
 * (levels outside 0..2), EUNSUPPORTED (levels > depth, depth > 3, levels =
 * 2 on an F64/I64 plan, or the deterministic combine mode), ENOMEM, ECUDA.
 * stark_plan_operands is not available in depth-first mode. */
STARK_API stark_status stark_plan_set_traversal(stark_plan_t plan, int levels);

/* Restrict the plan to the leaves [leaf_begin, leaf_end) of its recursion
 * tree, for sharding one product across devices (Stark runs the leaf
 * products as independent tasks spread over the cluster, Sec. III-C, Alg. 4;
 * its strong scaling over executors is Sec. V-F).  The workspace is
 * reallocated to hold only the operands of the subtrees below the top 2
 * recursion levels (1 for F64/I64) that contain those leaves, and
 * stark_mul_leaves on any sub-range of [leaf_begin, leaf_end) divides only
 * those subtrees (A and B read through the operand sums of the levels
 * above, formed on the fly as in the depth-first traversal) before its leaf
 * launch: a rank's divide work and workspace shrink with its share.
 * stark_mul on a restricted plan returns EINVAL (it is not the whole
 * product); [0, leaves) lifts the restriction.  Summing the partial C of
 * shards that partition [0, leaves) gives A*B.  Errors: EINVAL (empty or
 * out-of-range leaves), EUNSUPPORTED (depth > 3, depth 0, a depth-first
 * traversal, the K-major 3xTF32 layout), ENOMEM. */
STARK_API stark_status stark_plan_set_shard(stark_plan_t plan, int64_t leaf_begin, int64_t leaf_end);

/* Exact integer leaves on the tensor cores for an I64 plan whose inputs
 * satisfy |A_ij|, |B_ij| <= max_abs (the exact integer path;
 * the paper itself is FP64-only).  A depth-d leaf operand is a sum of 2^d
 * inputs, so with b = max_abs * 2^d the plan multiplies in bf16 (exact for
 * integers up to 256) with fp32 accumulation (exact while every partial sum
 * stays within 2^24) whenever b <= 256 and L * b^2 <= 2^24, and combines
 * into int64: bit-identical to the int64 CUDA-core path.  The divide checks
 * every operand on the device; a value beyond the range makes the next
 * stark_plan_check return STARK_EINVAL (the product is then invalid).
 * max_abs = 0 returns to the CUDA-core path.  Errors: EINVAL (not an I64
 * plan, max_abs < 0), EUNSUPPORTED (the bound does not give exactness at
 * this depth / leaf side; the plan keeps the CUDA-core path). */
STARK_API stark_status stark_plan_set_input_bound(stark_plan_t plan, int64_t max_abs);

/* Synchronise the plan's last stream and report any device-side error
 * recorded by its kernels since the previous check: STARK_ETIMEOUT for a
 * bounded wait that gave up, STARK_EINVAL for an integer operand outside the
 * bound declared with stark_plan_set_input_bound.  The error word is
 * cleared. */
STARK_API stark_status stark_plan_check(stark_plan_t plan, void *stream);

/* Per-phase device timing with CUDA events recorded on the product's own
 * stream.  stark_plan_set_timing(plan, k) pre-creates k event sets and
 * records the phases of the next k products (k = 0 switches timing off);
 * stark_plan_phase_ms waits for the last recorded product and returns the
 * mean over the recorded products of: [0] zeroing C, [1] divide A and B,
 * [2] leaf products with the fused combine.  Errors: EINVAL when nothing was
 * recorded. */
STARK_API stark_status stark_plan_set_timing(stark_plan_t plan, int records);
STARK_API stark_status stark_plan_phase_ms(stark_plan_t plan, float out_ms[3]);

/* The same means split one step further, `count` (1..4) of: [0] zeroing C,
 * [1] divide A and B, [2] the leaf-product kernel (with the fused combine,
 * when it is fused), [3] what follows it: the separate combine pass of
 * combine modes 2 and 3, the peeled edge and the staging copy into C (near 0
 * when there is none).  Errors: EINVAL when nothing was recorded or count is
 * out of range. */
STARK_API stark_status stark_plan_phases(stark_plan_t plan, float *out_ms, int count);

/* ----------------------------------------------------------------- batches */

typedef struct stark_batch_s *stark_batch_t;

/* A batch of `count` independent products C_i = A_i * B_i of sizes n[i] (any
 * mix), one tensor-core dtype (F32_SPLIT_BF16, F32_SPLIT_TF32 or
 * F32_SPLIT_FP16).  Every leaf
 * product of every member (Alg. 4) is a work item of ONE persistent grouped
 * leaf launch, whose epilogue combines (Alg. 5) into each member's own C;
 * the member divides (Alg. 3) precede it.  The launch sequence is recorded
 * in a CUDA graph on first use and replayed while the pointers stay the
 * same.  depth = -1: each member's depth and leaf tile are chosen by the
 * autotuner, which times the candidate (depth, tile) pairs on the device
 * (cached per size class and dtype for the process); otherwise members
 * whose leaf side allows it use 256-wide tiles.  Members on 256-wide tiles
 * share one grouped launch of CTA pairs, the others a second one with
 * 128-wide tiles on single CTAs.  Allocates every member's workspace.
 * Errors: EINVAL (count <= 0 or > 4096, n[i] <= 0, depth out of range),
 * EUNSUPPORTED (other dtypes, not a GB300), ENOMEM, ECUDA. */
STARK_API stark_status stark_batch_create(int32_t count, const int64_t *n, int depth, stark_dtype dtype,
                                          stark_batch_t *out);

/* Waits for the device, then frees everything the batch owns.  NULL is ignored. */
STARK_API stark_status stark_batch_destroy(stark_batch_t batch);

/* C[i] = A[i] * B[i] for every member.  A, B, C: host arrays of `count`
 * device pointers (member i is n[i] x n[i], row-major fp32).  Asynchronous
 * on `stream` (one graph launch); when any pointer differs from the previous
 * call the graph is re-recorded first, which waits for the device. */
STARK_API stark_status stark_batch_mul(stark_batch_t batch, const void *const *A, const void *const *B,
                                       void *const *C, void *stream);

/* Leaf tile width of member `index` (caller's order): 256 (CTA pairs on
 * 256 x 256 tiles) or 128 (single CTAs on 128 x 128 tiles); with depth -1
 * the autotuner times both where the leaf side allows 256 and keeps the
 * faster (with its depth). */
STARK_API stark_status stark_batch_tile(stark_batch_t batch, int32_t index, int32_t *tile_n);

/* Depth chosen for member `index`. */
STARK_API stark_status stark_batch_depth(stark_batch_t batch, int32_t index, int32_t *depth);

/* Widest leaf tile used (256 when any member runs 256-wide tiles), number of
 * grouped work items, device workspace bytes, and graph replays so far (any
 * pointer may be NULL). */
STARK_API stark_status stark_batch_info(stark_batch_t batch, int32_t *tile_n, int64_t *work_items,
                                        int64_t *workspace_bytes, int64_t *graph_replays);

/* Synchronise `stream` and report a device-side timeout of the batch's
 * kernels (STARK_ETIMEOUT), clearing it. */
STARK_API stark_status stark_batch_check(stark_batch_t batch, void *stream);

/* ----------------------------------------------------------------- serving */

typedef struct stark_server_s *stark_server_t;

/* Continuous-batching request server on the current device (the serving
 * form of the product; the paper has no serving layer).  One dispatcher
 * thread admits queued requests in arrival order while a stream slot is free
 * and their workspace fits `hbm_budget_bytes` (device bytes the server may
 * own for workspaces; idle workspaces are evicted least recently used first
 * to make room).  Each free slot takes a micro-batch of up to 16 admitted
 * requests and runs their divides plus ONE grouped leaf launch (as
 * stark_batch_mul), so requests arriving while others run overlap with them
 * on the device.  Workspaces are cached per padded size and stay resident.
 * A size whose breadth-first workspace (the operands of all 7^depth leaves)
 * exceeds the budget gets a depth-first workspace instead, holding the
 * operands of one subtree below the top 1 or 2 recursion levels (1/7 or 1/49
 * of the bytes; the fewest levels that fit; as stark_plan_set_traversal);
 * its requests run alone, subtree by subtree, not in the grouped launch.
 * When no traversal fits at the automatic depth, the fitting depth that the
 * cost model ranks fastest serves the request.  Thread-safe.  Errors: EINVAL (budget 0, slots outside 1..64),
 * EUNSUPPORTED, ENOMEM. */
STARK_API stark_status stark_server_create(size_t hbm_budget_bytes, int32_t slots, stark_server_t *out);

/* How a server with `hbm_budget_bytes` would hold a request of side n, on
 * the host alone (no device work): the recursion depth, the depth-first
 * levels of its workspace (0: breadth first; the limited-memory traversal
 * against the O(3^l N^2) space growth of Sec. VI) and the device bytes the
 * server counts against its budget for it: the leaf operand planes that the
 * divide (Alg. 3) writes for the 7^depth leaves of Alg. 1 (2 * 7^depth *
 * L^2 * 4 bytes for 3xBF16, * 8 for 3xTF32, F64, I64; L = n_pad / 2^depth),
 * divided by 7^levels, plus 1 MiB for the quadrant tables, plus the staging
 * copy of C (n_pad^2 * 4 bytes) when `staged` is non-zero and the dtype is a
 * split one (its C is one TMA cannot address: n % 4 != 0 or not 16-byte
 * aligned).  The depth is the cost model's choice, or the fitting depth the
 * cost model ranks fastest; for F64 and I64 that is the dispatcher's choice,
 * for the split dtypes the dispatcher tries its measured depth first.  Any
 * output pointer may be NULL.  ENOMEM: no depth fits (stark_submit refuses
 * such a request); EINVAL: n outside 0..2^20 or an unknown dtype. */
STARK_API stark_status stark_server_admission(size_t hbm_budget_bytes, int64_t n, stark_dtype dtype, int staged,
                                              int32_t *depth, int32_t *levels, int64_t *bytes);

/* Queue C = A*B (device pointers, n x n row-major, element type of dtype)
 * and return its id at once.  A, B, C must stay valid and unmodified until
 * stark_poll reports the request done.  ENOMEM: the request alone fits the
 * budget at no depth, even depth first (it could never be admitted); EINVAL:
 * bad arguments. */
STARK_API stark_status stark_submit(stark_server_t server, int64_t n, stark_dtype dtype, const void *A,
                                    const void *B, void *C, uint64_t *req_id);

/* Non-blocking: *done = 1 once the request finished (its status in
 * *req_status, if not NULL), else 0.  The poll that reports a request done
 * reaps it; later polls of that id return ENOTFOUND, as do unknown ids. */
STARK_API stark_status stark_poll(stark_server_t server, uint64_t req_id, int *done, stark_status *req_status);

/* Blocks until every submitted request finished (reaped or not). */
STARK_API stark_status stark_server_drain(stark_server_t server);

/* Latency of a finished request, in seconds from stark_submit until the
 * dispatcher observed its completion event.  EBUSY while it is pending,
 * ENOTFOUND for an unknown id. */
STARK_API stark_status stark_request_latency(stark_server_t server, uint64_t req_id, double *seconds);

/* Cached workspaces, device bytes they own, and requests waiting (any
 * pointer may be NULL). */
STARK_API stark_status stark_server_stats(stark_server_t server, int64_t *cached_workspaces, int64_t *owned_bytes,
                                          int64_t *queued);

/* Load counters since the server was created (any pointer may be NULL):
 * the most requests waiting in the queue at once, the requests whose
 * admission had to wait for device memory at least once (every workspace of
 * their size busy and no new one fitting the budget while others ran), and
 * the requests finished. */
STARK_API stark_status stark_server_load(stark_server_t server, int64_t *max_queued, int64_t *deferred,
                                         int64_t *finished);

/* Drains, stops the dispatcher and frees everything the server owns. */
STARK_API stark_status stark_server_destroy(stark_server_t server);

/* ----------------------------------------------------------------- no allocation */

/* Size of the fixed device scratch array behind stark_mul_noalloc. */
#define STARK_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* C = A * B for fp32 matrices with 3xBF16 leaves, like stark_mul on a plan of
 * dtype STARK_F32_SPLIT_BF16, but without allocating any device memory: for
 * callers that cannot call cudaMalloc (code that may not enter a memory
 * allocator, or that runs inside a fixed device-memory budget it may not
 * grow).  The paper has no counterpart; this is a deployment variant.
 *
 * The workspace is a file-scope device array of STARK_NOALLOC_SCRATCH_BYTES
 * (64 MiB) that every GPU which loads it keeps until the process exits.
 * Problems whose workspace does not fit are rejected with STARK_ENOMEM
 * (e.g. n <= 2048 fits at depth 0 or 1, n <= 1024 at depth 2).
 * A, B, C: device pointers to n x n row-major fp32 matrices; C is
 * overwritten.  depth: 0..3 (no automatic choice).  Asynchronous on
 * `stream`; nothing is allocated.  Each call rebuilds its C-target table in
 * the array with a kernel on `stream`, so no enqueued work reads host memory.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and must come before any stream capture.  Every
 * call reuses the same array: calls that overlap on the GPU (other streams
 * or threads) race and must be ordered by the caller.  A bounded device
 * wait that gave up is kept in the array's error word until
 * stark_noalloc_check reports it (later calls may then stop early too).
 * Errors: EINVAL (bad n or depth, null pointer), ENOMEM (over the scratch
 * size), EUNSUPPORTED (not a GB300), ECUDA. */
STARK_API stark_status stark_mul_noalloc(int64_t n, int depth, const void *A, const void *B, void *C,
                                         void *stream);

/* Synchronise `stream`, then report and clear a device-side timeout recorded
 * by stark_mul_noalloc calls on the current device since the last check
 * (STARK_ETIMEOUT: the products of those calls are invalid).  Allocates
 * nothing.  Errors: ECUDA. */
STARK_API stark_status stark_noalloc_check(void *stream);

/* ----------------------------------------------------------------- accuracy */

/* FP64 error statistics of a product, reduced on the device. */
typedef struct {
  double norm_a, norm_b;    /* ||A||_F, ||B||_F (sums of squares in fp64)                */
  double max_abs_err;       /* max |C_ij - ref_ij| over the compared entries              */
  double sum_sq_err;        /* sum (C_ij - ref_ij)^2                                       */
  double sum_sq_ref;        /* sum ref_ij^2 (relative RMS = sqrt(sum_sq_err / sum_sq_ref)) */
  double max_componentwise; /* max |C_ij - ref_ij| / absprod_ij over absprod_ij > 0        */
  int64_t compared;         /* entries compared: nrows * n                                 */
} stark_error_report;

/* The accuracy statement of a product on the device in FP64.  The paper runs
 * its products in FP64 and states no error (Sec. V); the split-precision
 * leaves are judged by the normwise ratio max|dC| / (||A||_F ||B||_F) and the
 * relative RMS error against FP64 reference rows, which this call reduces:
 * the Frobenius norms of A and B over all n^2 entries, and over `nrows`
 * sampled rows of C (row rows[r] of C against row r of `want`) the largest
 * absolute error, the sums of squares of the error and of the reference,
 * and, when `absprod` is not NULL, the largest componentwise ratio
 * |dC_ij| / (|A||B|)_ij.  Deterministic: fixed-order two-pass reductions.
 * A, B, C: device pointers to n x n row-major matrices of `dtype`'s element
 * type (fp32 for the split dtypes, fp64, int64 converted to fp64); rows:
 * device array of nrows row indices in [0, n); want, absprod: device arrays
 * of nrows x n fp64 (row-major).  nrows = 0 reduces the norms only (C, rows,
 * want may be NULL).  Synchronous on `stream`; allocates a few KB of device
 * memory per call.  Errors: EINVAL (bad sizes, NULL where data is needed),
 * ENOMEM, ECUDA. */
STARK_API stark_status stark_error_norms(int64_t n, stark_dtype dtype, const void *A, const void *B, const void *C,
                                         const int64_t *rows, int64_t nrows, const double *want,
                                         const double *absprod, stark_error_report *out, void *stream);

/* ----------------------------------------------------------------- tables */

/* The quadrant-index table ("block tags", Sec. III-B) for `depth` levels,
 * computed on the host; no device is needed.  For leaf l (base-7 M-index
 * path, top level most significant, so parent = l / 7 as in Alg. 5) and
 * side s (0: A-operand terms, 1: B-operand terms, 2: C targets), entries
 * [l*2^depth, l*2^depth + count[l]) of quad/sign list the quadrant paths q
 * (base-4, digit 0..3 = 11,12,21,22, top level most significant) and signs.
 * Arrays: count[7^depth], quad[7^depth * 2^depth], sign[7^depth * 2^depth]. */
STARK_API stark_status stark_quadrant_table(int depth, int side, int32_t *count, int32_t *quad, int8_t *sign);

/* ----------------------------------------------------------------- misc */

STARK_API const char *stark_strerror(stark_status status);

/* Self-check of the bounded device wait used by every kernel: launches one
 * tiny kernel that waits on a device flag nothing sets, with a limit of
 * `timeout_ns`, and synchronises.  Returns STARK_ETIMEOUT when the wait gave
 * up and reported it as designed (the CUDA context stays usable);
 * STARK_OK would mean the flag was seen set, which cannot happen. */
STARK_API stark_status stark_selftest_bounded_wait(uint64_t timeout_ns);

/* Number of kernels this library launched in this process so far. */
STARK_API int64_t stark_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* STARK_H */
