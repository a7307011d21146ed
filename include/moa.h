/*
 * moa.h — C ABI of libmoa, a GB300 (sm_103a) implementation of the
 * generalized inner and outer product of arbitrary-rank arrays from
 * Raynolds & Mullin, "A generalized inner and outer product of arbitrary
 * multi-dimensional arrays using A Mathematics of Arrays (MoA)".
 *
 * The paper's statement of the problem (Sec. I): every array is given to the
 * routine as a shape vector (rho A: the length of each axis) and a vector
 * holding its elements; both operations live behind one entry point that
 * takes a general binary operation.
 *
 *  - Outer product, Eq. (1): C_{ijkpqlm} = A_{ijkp} op B_{qlm};
 *    rho C = rho A ++ rho B.
 *  - Inner product, Eq. (2): D_{ijklm} = reduce_p ( A_{ijkp} combine B_{plm} );
 *    the last axis of A is contracted with the first axis of B,
 *    rho D = (rho A without its last axis) ++ (rho B without its first).
 *    (reduce, combine) = (add, mul) is matrix multiply (Sec. I).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Layout     Element vectors are row-major (C order) ravels of the array,
 *             as the appendix's addressing implies (element (i, p) of the
 *             flattened left operand at i*K + p, element (p, j) of the right
 *             operand and (i, j) of the result at p*N + j and i*N + j).
 *             MOA_B1_U32 arrays are
 *             the row-major ravel packed as a bit stream: element e is bit
 *             (e % 32) (LSB first) of 32-bit word e / 32; the last word's
 *             unused bits are zero on input and written as zero on output.
 *  Shapes     Host arrays of int64_t, read during the call only (the library
 *             keeps no pointer to them).  Entries must be >= 0, rank <= 8,
 *             and the element count must not overflow int64_t.
 *  Memory     A, B and out are device pointers owned by the caller, in
 *             memory of the current device (device or managed allocations;
 *             host memory or another GPU's memory returns
 *             MOA_ERR_NOT_DEVICE).  out
 *             holds prod(rho D) (inner) or prod(rho A)*prod(rho B) (outer)
 *             elements of out_dtype and must not overlap A or B.  The
 *             library owns only an internal scratch workspace, kept per
 *             (device, stream) and grown on demand with stream-ordered
 *             allocation; moa_release_workspace() frees it.
 *  Streams    Every call only enqueues work on `stream` (0 = legacy default
 *             stream) and returns; it never synchronises, except
 *             moa_device_status().  Calls that share a stream may share the
 *             workspace; calls on different streams never do.
 *  Errors     All arguments are validated on the host before any launch; a
 *             rejected call launches nothing and returns the error code.
 *             CUDA launch/API failures return MOA_ERR_CUDA.  Device-side
 *             waits are bounded: a kernel that gives up records
 *             MOA_ERR_TIMEOUT in a device status word that
 *             moa_device_status() reports.
 *  Exactness  Integer, min/max and Boolean results are bit-exact.  FP32
 *             single-operation results (semiring combine, outer product) are
 *             IEEE round-to-nearest-even, no flush-to-zero.  Floating (+,*)
 *             forms meet the normalised error |D - D_exact| / sum_p |A||B|
 *             stated beside moa_form.
 */
#ifndef MOA_H
#define MOA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (a CUDA stream handle); 0 is the default stream. */
typedef struct CUstream_st *moa_stream;

typedef enum {
    MOA_OK = 0,
    MOA_ERR_NULL = 1,           /* a required pointer is NULL */
    MOA_ERR_RANK = 2,           /* rank out of range for the operation */
    MOA_ERR_SHAPE_MISMATCH = 3, /* inner product with rho A[-1] != rho B[0] (Eq. 2) */
    MOA_ERR_OVERFLOW = 4,       /* negative extent, or an element count over int64 */
    MOA_ERR_UNSUPPORTED = 5,    /* (reduce, combine, dtype, form, out_dtype) not provided */
    MOA_ERR_WORKSPACE = 6,      /* scratch allocation failed */
    MOA_ERR_CUDA = 7,           /* a CUDA API call or launch failed */
    MOA_ERR_TIMEOUT = 8,        /* a device-side bounded wait gave up */
    MOA_ERR_INTERNAL = 9,
    MOA_ERR_ALIGNMENT = 10,     /* pointer not aligned to its element size */
    MOA_ERR_INVALID = 11,       /* malformed argument (e.g. bad enum, bad plan) */
    MOA_ERR_SCRATCH_LIMIT = 12, /* problem needs more scratch than the fixed no-allocation buffer holds */
    MOA_ERR_NOT_DEVICE = 13     /* A, B or out is not device memory of the current device */
} moa_status;

typedef enum {
    MOA_OP_ADD = 0,
    MOA_OP_SUB = 1,
    MOA_OP_MUL = 2,
    MOA_OP_DIV = 3,
    MOA_OP_MIN = 4,
    MOA_OP_MAX = 5,
    MOA_OP_OR = 6,
    MOA_OP_AND = 7
} moa_op;

/* Storage type of an element vector. */
typedef enum {
    MOA_F64 = 0,
    MOA_F32 = 1,
    MOA_BF16 = 2,
    MOA_FP8E4M3 = 3, /* OCP FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no infinities) */
    MOA_I32 = 4,
    MOA_B1_U32 = 5,  /* packed bits, see "Layout" above */
    MOA_F16 = 6      /* IEEE binary16 */
} moa_dtype;

/*
 * How the (add, mul) inner product is computed; other semirings take
 * MOA_FORM_NATIVE only.  Normalised error bounds (max over elements of
 * |D - D_exact| / sum_p |A||B|, D_exact from the operands as given):
 *   NATIVE    f64: FP64 FMA, <= 1e-12.  f32: FP32 FMA, <= 2e-6.
 *             i32: exact modulo 2^32.
 *             bf16, f16, fp8e4m3 (inputs already in that type; e4m3 with
 *             unit scales; FP32 out): tensor cores, one FP32 accumulator
 *             over the whole contraction (exact products, the running sum
 *             truncated at most once per 16-deep step), <= max(2e-6,
 *             (K/16) 2^-23) relative to the operands as given.
 *   BF16      f32 in/out: operands rounded to bf16, tensor cores, <= 1e-2.
 *   F16       f32 in/out: operands rounded to fp16 (RNE; magnitudes above
 *             65504 held at 65504), tensor cores, <= 2e-3 for operands
 *             whose magnitudes lie in fp16's normal range.
 *   FP8_T128  f32 in/out: operands scaled by powers of two per 1x128 block
 *             along the contraction and rounded to e4m3; tensor cores with
 *             the scale applied per block in FP32, <= 6e-2.
 *   BF16X3    f32 in/out: each operand split into three bf16 terms
 *             (hi + mid + lo), the six cross products of order <= 2
 *             accumulated in FP32 on tensor cores, <= 2e-6.
 *   OZAKI     f64 in/out: operands cut into fixed-point slices with
 *             per-row / per-column power-of-two exponents, exact slice
 *             products on tensor cores, recombined in FP64, <= 1e-12.
 *             Contraction length K <= 16384 (MOA_ERR_UNSUPPORTED beyond).
 */
typedef enum {
    MOA_FORM_NATIVE = 0,
    MOA_FORM_BF16 = 1,
    MOA_FORM_FP8_T128 = 2,
    MOA_FORM_BF16X3 = 3,
    MOA_FORM_OZAKI = 4,
    MOA_FORM_F16 = 5
} moa_form;

/*
 * moa_inner — generalized inner product, Eq. (2) (Sec. I):
 *   D[i.., j..] = reduce_{p=0}^{K-1} ( A[i.., p] combine B[p, j..] ),
 * folded from the identity of `reduce` (0 for add, +inf for min, -inf for
 * max, false for or).  K = rho A[rankA-1] = rho B[0]; K = 0 fills D with
 * that identity; an empty D is a no-op.  The arrays are flattened by psi
 * (Fig. 1: one result row per index vector of A's leading axes) into
 * M = prod(rho A[0..rankA-2]) rows, K, N = prod(rho B[1..rankB-1]) columns
 * without moving data.
 *
 * Supported (reduce, combine, dtype -> out_dtype, form):
 *   (add, mul) F64 -> F64      NATIVE | OZAKI
 *   (add, mul) F32 -> F32      NATIVE | BF16 | F16 | FP8_T128 | BF16X3
 *   (add, mul) BF16 -> F32     NATIVE
 *   (add, mul) F16 -> F32      NATIVE
 *   (add, mul) FP8E4M3 -> F32  NATIVE (no NaN inputs)
 *   (add, mul) I32 -> I32      NATIVE (wraps modulo 2^32; when every value lies in
 *                              [-128, 127] and K <= 1024 it runs on tensor cores,
 *                              with the same bits)
 *   (min|max, add|sub|mul|min|max) F32 -> F32   NATIVE
 *       ((min, add) shortest paths, (max, min) widest paths, (min, max)
 *       minimax paths, ...; NaN counts as missing, as C's fminf / fmaxf)
 *   (or, and) B1_U32 -> B1_U32      NATIVE (tensor cores by exact counting when
 *                                   M, N > 128 and N % 32 == 0)
 * rankA, rankB in [1, 8].  Returns MOA_ERR_SHAPE_MISMATCH when
 * rho A[-1] != rho B[0], MOA_ERR_UNSUPPORTED for any other tuple.
 */
moa_status moa_inner(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                     const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB, const void *B,
                     void *out, moa_dtype out_dtype, moa_stream stream);

/*
 * moa_inner_host — moa_inner for arrays held in host memory: the same
 * Eq. (2), tuples, forms, exactness and errors, with A, B and out host
 * pointers (page-locked memory, e.g. from cudaHostAlloc, lets the copies
 * run asynchronously; pageable memory works but the copies then wait for
 * the host).  The call enqueues on `stream` the copy of B and A to the
 * device, the inner product, and the copy of D back into out; when D has
 * more than 1024 rows (psi-flattened M), its rows are computed in up to four
 * blocks so that the copies of one block overlap the computation of
 * another (library-owned copy streams, ordered with `stream` by events).
 * The host buffers must stay valid and unchanged until `stream` reaches the
 * end of the call.  Device copies live in a library workspace kept per
 * (device, stream) (MOA_ERR_WORKSPACE when it cannot be had).  A device
 * pointer for A, B or out returns MOA_ERR_INVALID.
 */
moa_status moa_inner_host(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                          const int64_t *shapeA, const void *A, int rankB, const int64_t *shapeB, const void *B,
                          void *out, moa_dtype out_dtype, moa_stream stream);

/*
 * moa_inner_e4m3_scaled — the (add, mul) inner product, Eq. (2) in its
 * matrix-multiply case (Sec. I), of FP8 E4M3 arrays stored with per-block
 * power-of-two scales, the layout of MOA_FORM_FP8_T128:
 *   A[i.., p] = a8[i.., p] * scale_a[i][p / 128],
 *   B[p, j..] = b8[p, j..] * scale_b[p / 128][j / 128]   (psi-flattened i, j),
 *   D = A . B in FP32 (tensor cores, one FP32 accumulator over the whole
 *   contraction; normalised error <= max(2e-6, (K/16) 2^-23) relative to the
 *   scaled operands).
 * scale_a: M x ceil(K/128) FP32, scale_b: ceil(K/128) x ceil(N/128) FP32,
 * row-major device memory of the current device.  Each scale is used as the
 * power of two of its exponent field (2^floor(log2 |s|)); scales should be
 * finite normal powers of two.  Shapes, errors and streams as for moa_inner
 * with dtype MOA_FP8E4M3; a NULL scale array returns MOA_ERR_NULL.
 */
moa_status moa_inner_e4m3_scaled(int rankA, const int64_t *shapeA, const void *A, const float *scale_a, int rankB,
                                 const int64_t *shapeB, const void *B, const float *scale_b, float *out,
                                 moa_stream stream);

/*
 * moa_inner_axes — Eq. (2) contracting axis `axisA` of A with axis `axisB`
 * of B (equal lengths) instead of A's last and B's first:
 *   D[i.., j..] = reduce_p ( A[.., p at axisA, ..] combine B[.., p at axisB, ..] ),
 *   rho D = (rho A without axisA) ++ (rho B without axisB).
 * Equals moa_inner on A transposed to move axisA last and B transposed to
 * move axisB first (moa_transpose below, into a library workspace of those
 * sizes kept per stream; MOA_ERR_WORKSPACE when it cannot be had).  Same tuples, forms, errors and exactness as moa_inner;
 * 0 <= axisA < rankA and 0 <= axisB < rankB, else MOA_ERR_INVALID.  Packed
 * Booleans are supported only where no transpose is needed.
 */
moa_status moa_inner_axes(moa_op reduce, moa_op combine, moa_dtype dtype, moa_form form, int rankA,
                          const int64_t *shapeA, const void *A, int axisA, int rankB, const int64_t *shapeB,
                          const void *B, int axisB, void *out, moa_dtype out_dtype, moa_stream stream);

/*
 * moa_transpose — out = A with its axes permuted: output axis k is input
 * axis perm[k], rho out[k] = rho A[perm[k]] (both row-major element
 * vectors).  rank in [0, 8]; perm a permutation of 0..rank-1, else
 * MOA_ERR_INVALID; dtype any but MOA_B1_U32 (MOA_ERR_UNSUPPORTED); out must
 * not overlap A.  Bit-exact data movement; asynchronous on `stream`.
 */
moa_status moa_transpose(moa_dtype dtype, int rank, const int64_t *shape, const int *perm, const void *A, void *out,
                         moa_stream stream);

/*
 * moa_outer — generalized outer product, Eq. (1) (Sec. I; the operator of
 * the outer product may be any binary operation, + - * / among them):
 *   C[i.., j..] = A[i..] op B[j..],  rho C = rho A ++ rho B.
 * Supported (op, dtype -> out_dtype):
 *   add|sub|mul|div|min|max: F64 -> F64, F32 -> F32,
 *                            BF16 -> BF16 (op in FP32, rounded once, RNE),
 *                            BF16 -> F32;
 *   add|sub|mul:             I32 -> I32 (wraps modulo 2^32).
 * rankA, rankB in [0, 8] (a rank-0 operand is a scalar).
 */
moa_status moa_outer(moa_op op, moa_dtype dtype, int rankA, const int64_t *shapeA, const void *A, int rankB,
                     const int64_t *shapeB, const void *B, void *out, moa_dtype out_dtype, moa_stream stream);

/*
 * moa_inner_shape — rho D of Eq. (2) without computing anything; the Fig. 1
 * example rho A = <2 3>, rho B = <3 4> gives rho D = <2 4>.  shapeD must hold
 * rankA + rankB - 2 entries.  Pure host function.
 */
moa_status moa_inner_shape(int rankA, const int64_t *shapeA, int rankB, const int64_t *shapeB, int *rankD,
                           int64_t *shapeD);

/* moa_outer_shape — rho C = rho A ++ rho B (Eq. 1); shapeC holds rankA + rankB entries. */
moa_status moa_outer_shape(int rankA, const int64_t *shapeA, int rankB, const int64_t *shapeB, int *rankC,
                           int64_t *shapeC);

/* ------------------------------------------------------------- batching */

/*
 * One problem of a batch: an inner product (kind 0) or an outer product
 * (kind 1), described exactly as for moa_inner / moa_outer.  The shape
 * arrays are read during moa_batch_plan_create only; A, B and out are device
 * pointers that must stay valid, and keep their sizes, for every execute.
 */
typedef struct {
    int32_t kind; /* 0 inner (Eq. 2), 1 outer (Eq. 1) */
    int32_t reduce;   /* moa_op; inner only */
    int32_t combine;  /* moa_op; the op of an outer product */
    int32_t dtype;    /* moa_dtype of A and B */
    int32_t form;     /* moa_form; inner (add, mul) only */
    int32_t out_dtype;
    int32_t rankA, rankB;
    const int64_t *shapeA;
    const int64_t *shapeB;
    const void *A;
    const void *B;
    void *out;
} moa_problem;

typedef struct moa_batch_plan moa_batch_plan;

/*
 * moa_batch_plan_create — validate `count` problems (each as its single call
 * would), cut them into work items (128 x 128 tiles of inner products, row
 * blocks of outer products), lay out the device descriptor array, the item
 * queues, the split-plane scratch and the tensor maps, and allocate the
 * plan's own device memory on the current device.  On error nothing is left
 * allocated and *plan is NULL; the index of the first bad problem is written
 * to *bad_index (if not NULL).  Supported problems: (add, mul) F32 with forms
 * BF16X3 or NATIVE; (min|max, add|mul) F32; outer F32 ops.
 */
moa_status moa_batch_plan_create(int count, const moa_problem *problems, moa_batch_plan **plan, int *bad_index);

/*
 * moa_batch_execute — run every problem of the plan on `stream`.  The first
 * execute times the plan's schedules on `stream` (the choice is cached per
 * GPU and plan signature in $MOA_TUNE_CACHE, default
 * ~/.cache/moa_autotune.txt; MOA_AUTOTUNE=off|cached|force,
 * MOA_BATCH_SCHEDULE=0..15 fixes one) and records the chosen launch
 * sequence into a CUDA graph; every execute then launches that graph on
 * `stream`.  Problems write disjoint outputs.
 */
moa_status moa_batch_execute(moa_batch_plan *plan, moa_stream stream);

/* Plan statistics: problem count, kernels per execute (of the chosen schedule; before the first execute, of the
 * default one), total work items, total flop-equivalent work. */
moa_status moa_batch_plan_info(const moa_batch_plan *plan, int64_t *n_problems, int64_t *n_launches,
                               int64_t *n_tiles, double *work_flops);

/* Release the plan (synchronises the device first). NULL is accepted. */
void moa_batch_plan_destroy(moa_batch_plan *plan);

/* ------------------------------------------------------------ utilities */

/* Human-readable name of a status code (static string). */
const char *moa_status_string(moa_status s);

/*
 * moa_device_status — synchronise `stream`, then read and clear the device
 * status word written by bounded waits; returns MOA_ERR_TIMEOUT if any
 * kernel gave up since the last call, MOA_ERR_CUDA on a sticky CUDA error,
 * MOA_OK otherwise.
 */
moa_status moa_device_status(moa_stream stream);

/*
 * moa_selftest_wait_timeout — exercise the bounded-wait machinery: launch one
 * CTA that waits on a barrier nothing ever completes, for limit_us
 * microseconds (1 .. 1,000,000), after which it gives up and records a
 * time-out, so the next moa_device_status() returns MOA_ERR_TIMEOUT and the
 * context stays usable.  Diagnostic only (no counterpart in the paper).
 */
moa_status moa_selftest_wait_timeout(uint32_t limit_us, moa_stream stream);

/*
 * moa_kernel_timing — diagnostic timing of the library's tensor-core GEMM
 * launches (no counterpart in the paper): with enable = 1 every such launch
 * on the current device is bracketed by a pair of CUDA events recorded on
 * its stream (and the record of an earlier start is cleared); enable = 0
 * stops recording.  moa_kernel_timing_read waits for the recorded events and
 * returns how many launches were recorded and their summed device time in
 * milliseconds.  Other kernels (pre-passes, CUDA-core kernels) are not
 * recorded.
 */
moa_status moa_kernel_timing(int enable);
moa_status moa_kernel_timing_read(int64_t *launches, double *total_ms);

/*
 * moa_ozaki_slices — the number of digit slices per operand the OZAKI form
 * takes for a contraction of length K (its slice-pair GEMM does
 * S (S + 1) / 2 products), after any MOA_OZAKI_SLICES override; 0 for
 * K < 0.  Host-side query, no device work.  Diagnostic only (no counterpart
 * in the paper).
 */
int moa_ozaki_slices(int64_t K);

/* Free the scratch workspace held for every stream of the current device (synchronises). */
moa_status moa_release_workspace(void);

/* Library version, e.g. 0x000100 for 0.1.0. */
int moa_version(void);

/* ------------------------------------------------ no-allocation variant */

/* Size of the fixed scratch buffer used by moa_inner_bf16x3_noalloc. */
#define MOA_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/*
 * moa_inner_bf16x3_noalloc — the (add, mul) inner product of FP32 arrays in
 * the split-BF16x3 form (same result as moa_inner(MOA_OP_ADD, MOA_OP_MUL,
 * MOA_F32, MOA_FORM_BF16X3, ..., MOA_F32, stream)), for callers that must not
 * allocate device memory.  The paper has no counterpart to this call: it
 * exists for the library's users, not for the method.
 *
 * Who needs it: code that runs where an allocation is not allowed or not
 * affordable — inside a region being captured into a CUDA graph (a
 * cudaMalloc there breaks or invalidates the capture), a serving loop with
 * a fixed memory budget that must never grow or stall on the allocator
 * (cudaMalloc can synchronise the device), or a host callback / custom
 * allocator hook where calling back into an allocator is not permitted.
 *
 * Scratch: the bf16 split planes live in one file-scope device array of
 * MOA_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library
 * holds until the process exits.  A problem needs 6 * (M*Kp + K*Np) bytes,
 * Kp and Np being K and N rounded up to a multiple of 8 (M, K, N the
 * psi-flattened extents, as for moa_inner); a larger one returns
 * MOA_ERR_SCRATCH_LIMIT before any launch.  Nothing in the array needs to
 * start at zero (every byte a call reads is written earlier in that call).
 *
 * Set-up: the first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, no allocation) with that device current;
 * make that first call before any stream capture.  The call allocates
 * nothing — no cudaMalloc, cudaFree or allocating library routine.
 *
 * Concurrency: every call shares the one array, so calls that can overlap
 * on the GPU (different streams, or different host threads) race; serialise
 * them, e.g. on one stream.  Arguments, validation and errors otherwise as
 * for moa_inner.
 */
moa_status moa_inner_bf16x3_noalloc(int rankA, const int64_t *shapeA, const float *A, int rankB,
                                    const int64_t *shapeB, const float *B, float *out, moa_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MOA_H */
