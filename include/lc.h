/*
 * lc.h -- C ABI of the GB300 (sm_103a) batched element-local contraction library.
 *
 * The computation is the dG FEM volume workload of Table 1:
 *
 *     out[f, e, i] = sum_j D[f, i, j] * u[e, j]
 *         over the loop domain { [f,e,i,j] : 0<=f<F and 0<=e<E and 0<=i,j<N }
 *
 * stated, as in Section 2.1, as a loop domain plus one instruction with a sum
 * reduction, plus optional assumptions on the parameters.  The transformations
 * of Section 2.4 (split_iname of Eq. 1 with tail guards, the unr / ilp / vec
 * iname tags, array-axis layout tags, add_prefetch / precompute) are not applied
 * by a code generator here: each is a field of an explicit variant descriptor
 * (lc_variant) that selects a hand-written CUDA kernel instance.  Every variant
 * computes the same result up to rounding (the unordered semantics of
 * Section 2.3).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers; the caller allocates and owns
 *     them.  The library never allocates device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously, like the event-returning invocation of
 *     Section 2.2; argument errors are returned before anything is enqueued.
 *   - Arrays are dense and row-major:
 *       D    [F][N][N]               D[(f*N + i)*N + j]
 *       u    element-major [E][N]    u[e*N + j]        node-major [N][E]  u[j*E + e]
 *       out  element-major [F][E][N]                   node-major [F][N][E]
 *     Element type: double for LC_PREC_FP64, float for every other precision.
 *   - All entry points are thread-safe; a kernel handle is immutable after
 *     creation (Section 2.4: transformations return new kernels).
 *   - Per-device state (the device error word, the copy streams of lc_contract_host,
 *     the address of lc_error_norm_noalloc's array) is looked up once per device and
 *     kept for the life of the process: do not use the library across a
 *     cudaDeviceReset of a device it has already run on.
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lc_status {
    LC_OK = 0,
    LC_ERR_INVALID_ARGUMENT = 1, /* null pointer, negative size, bad enum value */
    LC_ERR_UNSUPPORTED = 2,      /* domain / instruction / assumption text not recognised */
    LC_ERR_INVALID_VARIANT = 3,  /* descriptor fields out of range for this problem */
    LC_ERR_ASSUMPTION = 4,       /* E, N, F violate the kernel's assumptions */
    LC_ERR_MISALIGNED = 5,       /* a pointer is not aligned as the variant needs */
    LC_ERR_BUFFER_TOO_SMALL = 6, /* caller buffer (text or workspace) too small */
    LC_ERR_CUDA = 7,             /* a CUDA runtime call failed; see lc_last_cuda_error */
    LC_ERR_TIMEOUT = 8,          /* a bounded device wait gave up (device error word) */
    LC_ERR_NO_DEVICE = 9,        /* no sm_103 device current */
    LC_ERR_NOT_FOUND = 10,       /* lookup failed (e.g. no timing for a candidate) */
    LC_ERR_INDEX = 11            /* an index array held an entry out of range (device error word) */
} lc_status;

/* Human-readable name of a status. Never NULL. */
const char *lc_status_string(lc_status s);
/* The last CUDA error code seen by this thread (0 if none). */
int lc_last_cuda_error(void);

/* ------------------------------------------------------------------------- */
/* Kernel: loop domain + instruction + assumptions (Section 2.1).            */
/* ------------------------------------------------------------------------- */
typedef struct lc_kernel lc_kernel;
typedef struct lc_variant lc_variant;

/*
 * Parse and validate a contraction kernel.
 *   domain       isl-style set, e.g. "{ [f,e,i,j]: 0<=f<F and 0<=e<E and 0<=i,j<N }".
 *                Every iname must have lower bound 0 and an upper bound "< P" or
 *                "<= P - 1" with P a parameter name.  A three-iname domain
 *                "{ [e,i,j]: ... }" is the single-operator form (F = 1).
 *   instructions one assignment "out[f,e,i] = sum(j, D[f,i,j]*u[e,j])" (names are
 *                free; the index structure must be this one, factors in either
 *                order; single-operator form "out[e,i] = sum(j, D[i,j]*u[e,j])").
 *   assumptions  NULL or a conjunction of "P mod k = 0", "P >= k", "P > k",
 *                "P <= k", "P < k", "P = k" over the domain's parameters.
 *   out          receives a new handle (free with lc_kernel_destroy).
 * Errors: LC_ERR_INVALID_ARGUMENT (null text/out), LC_ERR_UNSUPPORTED (text
 * outside the forms above; *out is left untouched).
 */
lc_status lc_kernel_create(const char *domain, const char *instructions,
                           const char *assumptions, lc_kernel **out);
void lc_kernel_destroy(lc_kernel *k);

/*
 * Text dump of a kernel in the spirit of Section 2.1's listing: arguments with
 * shapes and dimension tags, domain, assumptions, instruction; with a variant,
 * also the transformations it applies (split of e with its guard, iname tags,
 * layout tags, prefetch).  Writes at most `cap` bytes including the NUL; sets
 * *needed to the full length + 1.  `v` may be NULL.
 * Errors: LC_ERR_BUFFER_TOO_SMALL (text truncated, still NUL-terminated).
 */
lc_status lc_kernel_print(const lc_kernel *k, const lc_variant *v, char *buf,
                          size_t cap, size_t *needed);

/* ------------------------------------------------------------------------- */
/* Variant descriptor (the transformations of Section 2.4 as values).        */
/* ------------------------------------------------------------------------- */
enum { LC_ENGINE_SIMT = 0, LC_ENGINE_TCGEN05 = 1, LC_ENGINE_WARP = 2, LC_ENGINE_KSPLIT = 3 };
enum { LC_LAYOUT_ELEM_MAJOR = 0, LC_LAYOUT_NODE_MAJOR = 1 };
enum { LC_PREC_FP64 = 0, LC_PREC_FP32 = 1, LC_PREC_BF16 = 2, LC_PREC_BF16X3 = 3 };

struct lc_variant {
    uint32_t struct_size;     /* sizeof(lc_variant) */
    int32_t engine;           /* LC_ENGINE_*: SIMT FMA tiles, tcgen05 tensor cores, one warp
                                 per element group with shuffles (small N), or K-split SIMT
                                 (FP32): 8 x 8 register blocks over a tile_e x 128 output
                                 block, the j reduction cut into chunks of `unroll` (8 or 16)
                                 whose D^T rows are fetched one chunk ahead, so D^T need not
                                 fit in shared memory; tile_e 64 or 128, elems_per_thread =
                                 split_i = 8, prefetch_smem 1, stages = u tile buffers (1, 2) */
    int32_t layout;           /* LC_LAYOUT_*: array-axis layout tag of u and out (Sec. 2.4.3) */
    int32_t precision;        /* LC_PREC_*: FP64/FP32 on the FMA pipes; BF16 or three-term
                                 split BF16 on the tensor cores with FP32 accumulation */
    int32_t tile_e;           /* split_iname(e, tile_e): e = e_in + tile_e * e_out (Eq. 1),
                                 one tile per CTA step */
    int32_t elems_per_thread; /* ilp tag on e_in: elements per thread (SIMT register block);
                                 tensor-core engine: K-block width of the shared-memory
                                 operands, 16, 32 or 64 (1 = widest dividing N rounded to 16) */
    int32_t split_i;          /* ilp tag on i: output columns per thread (SIMT register block);
                                 tensor-core engine: operators per CTA column block (0 = most) */
    int32_t unroll;           /* unr tag on the j reduction: 1, 2, 4 or 8; tensor-core engine:
                                 epilogue threads per tile row, 1 to 4 (conversion threads per
                                 row: the same, 2 for 4) */
    int32_t prefetch_smem;    /* add_prefetch of the u tile into shared memory by TMA (1) or
                                 direct global loads into registers (0); tensor-core engine: 1,
                                 or 2 = each converting thread takes its values into registers,
                                 splits them into their bf16 terms and frees the stage at once,
                                 so only its stores wait for the A buffer (K of one block, at
                                 most 3 chunks of 8 nodes a thread for BF16, 2 for BF16X3;
                                 others take the plain path) */
    int32_t tail_free;        /* 1: no guard on the last e tile; only accepted when an
                                 assumption "E mod m = 0" with m a multiple of tile_e holds */
    int32_t stages;           /* u tiles in flight in shared memory (TMA ring depth), >= 1 */
    int32_t ctas_per_sm;      /* persistent grid size in CTAs per SM; 0 = one CTA per tile */
    int32_t out_buffers;      /* tensor-core engine, element-major: shared-memory staging slots of
                                 one operator's output tile each, whose bulk stores may be in
                                 flight together (1 to 4; 0 = the planner's choice) */
    int32_t store_rows;       /* tensor-core engine, element-major: tile rows written by one bulk
                                 store: 32 or 64 (the warps of 1 or 2 TMEM lane quarters stage
                                 one operator at a time and store it), or 128 (all epilogue
                                 warps stage every operator of the block, then store);
                                 0 = the planner's choice */
    int32_t max_ctas;         /* upper bound on the persistent grid (0 = none): the CTAs then
                                 walk more tiles each, and the rest of the GPU stays free for
                                 concurrent work; at least the number of column blocks */
    int32_t mma_order;        /* tensor-core engine, BF16X3: 0 = the planner's choice, 1 = the
                                 large hi*hi products in their own accumulator columns (two D
                                 terms stacked along the MMA's N), 2 = one accumulator, the
                                 small products first over all of K and hi*hi last; must be 0
                                 for other paths */
    int32_t a_operand;        /* tensor-core engine: where the converted u tile (the MMA's A
                                 operand) lives: 0 = the planner's choice, 1 = shared memory,
                                 2 = tensor memory beside the accumulators, written by the
                                 conversion warps with tcgen05.st: frees shared memory and its
                                 bandwidth (BF16X3: one accumulator region per buffer, the
                                 products unstacked; the planner takes it where no shared-
                                 memory plan fits, N up to 128; not for the three-term
                                 geometric-factor kernel) */
};

/*
 * A reasonable descriptor for (E, N, F, layout, precision): fills *v.  The choices follow
 * the autotuner's measurements on this GPU: FP32 on the warp engine up to N = 12, SIMT
 * tiles below N = 96, the K-split engine from N = 96; BF16 and BF16X3 on the tensor cores
 * (BF16X3 with the A terms in shared memory, from about N = 100 to 128 in tensor memory),
 * and where no tensor-core plan exists the FP32 kernels, whose error is below both
 * reduced-precision bounds; FP64 SIMT tiles.  No GPU work is done.
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_UNSUPPORTED (no engine supports it).
 */
lc_status lc_variant_default(const lc_kernel *k, int64_t E, int32_t N, int32_t F,
                             int32_t layout, int32_t precision, lc_variant *v);

/*
 * Check a descriptor against a problem size without launching anything:
 * field ranges, shared-memory capacity, assumption-gated fast paths.
 * Errors: LC_ERR_INVALID_VARIANT, LC_ERR_ASSUMPTION, LC_ERR_INVALID_ARGUMENT.
 */
lc_status lc_variant_validate(const lc_kernel *k, int64_t E, int32_t N, int32_t F,
                              const lc_variant *v);

/*
 * The launch plan a valid descriptor resolves to for a problem size: what the split,
 * ilp and prefetch transformations of Section 2.4 amount to on this GPU (the CUDA
 * device current on the calling thread; without one, a 148-SM, 227 KB part is assumed).
 * Nothing is launched.  The caller sets p->struct_size = sizeof(lc_plan).
 * Errors: those of lc_variant_validate; LC_ERR_INVALID_ARGUMENT for a null or
 * mis-sized p; LC_ERR_UNSUPPORTED for a surface-lift kernel (its plan depends on the
 * face counts, which this call does not take).
 */
typedef struct lc_plan {
    uint32_t struct_size;    /* sizeof(lc_plan) */
    int32_t grid;            /* CTAs launched */
    int32_t threads;         /* threads per CTA */
    int32_t smem_bytes;      /* dynamic shared memory per CTA */
    int64_t tiles;           /* element tiles (ceil(E / tile)) */
    int32_t column_blocks;   /* CTAs that share one element tile (operator or row blocks) */
    int32_t ops_per_block;   /* operators per column block (0: blocks are row ranges) */
    /* tensor-core engine only (0 otherwise) */
    int32_t k_mma;           /* K the MMAs read: N rounded up to 16 */
    int32_t k_block;         /* K-block width (bf16 values per swizzled row) */
    int32_t cols_per_op;     /* accumulator columns per operator */
    int32_t mma_n;           /* MMA N: accumulator columns per column block */
    int32_t stacked;         /* 1: BF16X3 D terms stacked along N (5 MMAs per K step, not 6) */
    int32_t a_buffers;       /* A-operand buffers */
    int32_t out_slots;       /* element-major output staging slots */
    int32_t store_rows;      /* element-major tile rows per bulk store */
    int32_t mma_per_tile;    /* tcgen05.mma instructions per tile and column block */
    int32_t a_in_tmem;       /* 1: the A terms live in tensor memory */
    int32_t tmem_cols;       /* tensor-memory columns allocated per CTA */
} lc_plan;

lc_status lc_variant_plan(const lc_kernel *k, int64_t E, int32_t N, int32_t F, const lc_variant *v,
                          lc_plan *p);

/*
 * The contraction itself: enqueue out = contraction(D, u) on `stream`.
 *   D_dev    [F][N][N] operators (double for FP64, else float)
 *   u_dev    input, layout per v->layout
 *   out_dev  output, layout per v->layout; must not overlap u_dev or D_dev
 * Sizes: E >= 0, 1 <= N <= 256, 1 <= F <= 8.  E == 0 enqueues nothing.
 * Alignment: every pointer 16-byte aligned.
 * Errors (returned before any launch): LC_ERR_INVALID_ARGUMENT, LC_ERR_INVALID_VARIANT,
 * LC_ERR_ASSUMPTION, LC_ERR_MISALIGNED, LC_ERR_NO_DEVICE; launch failures: LC_ERR_CUDA.
 * Bounded device waits that give up set the device error word (lc_device_error).
 */
lc_status lc_contract(const lc_kernel *k, const lc_variant *v, const void *D_dev,
                      const void *u_dev, void *out_dev, int64_t E, int32_t N, int32_t F,
                      void *stream);

/* ------------------------------------------------------------------------- */
/* General front end: elementwise instructions (Section 2.1, 2.4).            */
/* ------------------------------------------------------------------------- */
/*
 * A kernel whose domain has one or two inames, e.g. "{ [i]: 0<=i<n }" or
 * "{ [i,j]: 0<=i<n and 0<=j<m }", and whose instruction is one assignment
 *     out[i] = expr        or        out[i,j] = expr
 * with expr built from +, -, *, / (usual precedence, left to right), unary minus,
 * parentheses, decimal literals, scalar parameters (names without an index) and array
 * accesses indexed by the domain's inames in domain order (a subset of them: "c[j]" inside
 * [i,j] is broadcast along i).  The saxpy of Table 1 is "z[i] = a*x[i] + y[i]".
 *
 * lc_elementwise generates a CUDA kernel for the instruction (once per instruction,
 * unroll factor and edge handling; compiled for this GPU at run time with NVRTC and cached
 * for the life of the process) and launches it.  The transformations of Section 2.4 are
 * the descriptor's fields: split_iname of the innermost iname into tiles (256 x 4 x unroll
 * elements for one iname; 256 columns x 4 x unroll rows for two), bulk tiles with no guard
 * and 16-byte vectors (elems_per_thread 4; 1 = scalar code throughout), separate edge code
 * for tiles cut by one bound and corner code for tiles cut by both, chosen per tile at run
 * time; tail_free = 1 drops the edge code when an assumption "n mod tile = 0" holds (one
 * iname only).  Every operation is one IEEE binary32 operation rounded to nearest, never
 * contracted into a fused multiply-add: the result is the plain loop's, bit for bit.
 * Descriptor: engine SIMT, precision FP32, element-major layout, unroll 1/2/4/8,
 * elems_per_thread 1 or 4, ctas_per_sm (0 = 4), max_ctas, tail_free; every other field 0
 * (stages 1); tile_e 0 or the tile above.  lc_variant_default gives unroll 4, vectors,
 * 4 CTAs per SM; lc_variant_validate and lc_variant_plan take the extents of the first and
 * second iname as E and N (N ignored for one iname) and F = 1.
 */

/* Argument counts of a kernel: arrays (elementwise: the output, then the inputs in order
 * of first appearance; contraction: out, D, u; volume derivative: out, D, u, G), scalar
 * parameters (in order of first appearance) and domain inames. */
lc_status lc_kernel_signature(const lc_kernel *k, int32_t *n_arrays, int32_t *n_params, int32_t *n_dims);

/* The name of argument `index` of kind `what` (0 array, 1 scalar parameter, 2 the bound
 * of iname `index`), NUL-terminated in buf[cap].  Errors: LC_ERR_INVALID_ARGUMENT (no such
 * argument), LC_ERR_BUFFER_TOO_SMALL (truncated). */
lc_status lc_kernel_arg_name(const lc_kernel *k, int32_t what, int32_t index, char *buf, size_t cap);

/* The CUDA source lc_elementwise would compile for (v, extents), NUL-terminated in
 * buf[cap]; *needed = its length + 1.  Nothing is compiled or launched. */
lc_status lc_elementwise_source(const lc_kernel *k, const lc_variant *v, const int64_t *extents, char *buf,
                                size_t cap, size_t *needed);

/*
 * Enqueue the elementwise instruction over the domain on `stream`.
 *   extents     one per iname, in domain order (>= 0)
 *   arrays_dev  one device pointer per array in signature order (arrays_dev[0] = the
 *               output); float, dense row-major over the inames each array is indexed by;
 *               4-byte aligned, 16-byte aligned for the vector code (elems_per_thread 4 and,
 *               with two inames, the inner extent a multiple of 4); the output must not
 *               overlap an input
 *   params      one value per scalar parameter, in signature order (rounded to binary32)
 * The first call for a new instruction compiles it (NVRTC; synchronous, tens of
 * milliseconds): make it before any stream capture.
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_INVALID_VARIANT, LC_ERR_ASSUMPTION,
 * LC_ERR_MISALIGNED, LC_ERR_NO_DEVICE, LC_ERR_UNSUPPORTED (not an elementwise kernel, or
 * no run-time compiler on this machine), LC_ERR_CUDA.
 */
lc_status lc_elementwise(const lc_kernel *k, const lc_variant *v, const int64_t *extents, void *const *arrays_dev,
                         const double *params, void *stream);

/*
 * The volume derivative with per-element geometric factors: the dG FEM volume workload of
 * Table 1 with the chain rule applied inside the kernel,
 *
 *     out[d, e, i] = sum_f r[e, d, f] * sum_j D[f, i, j] * u[e, j]      d, f < F
 *
 * stated to lc_kernel_create as the domain { [d,f,e,i,j] : 0<=d<F and 0<=f<F and 0<=e<E and
 * 0<=i,j<N } and the instruction "out[d,e,i] = sum((f,j), G[e,d,f]*D[f,i,j]*u[e,j])" (the
 * three factors in any order).  The F reference derivatives of a node stay in tensor memory;
 * the epilogue mixes them with the element's F x F factors (FP32) before the one store, so
 * the output is written once instead of twice, and the F partial results never reach memory.
 * Tensor-core engine only (LC_PREC_BF16, or LC_PREC_BF16X3 for FP32-level accuracy), F = 2
 * or 3, every operator in one column block (split_i 0 or F), element-major store_rows 0 or
 * 128.  The accumulators of all F operators and a whole-tile staging slot of F outputs must
 * fit one SM: element-major BF16X3 plans exist up to N = 48 for F = 3 and N = 64 for F = 2
 * (lc_variant_default returns LC_ERR_UNSUPPORTED beyond).
 *   D_dev    [F][N][N] float       u_dev  layout per v->layout
 *   r_dev    element-major [E][F][F] (r[(e*F + d)*F + f]); node-major [F][F][E]
 *   out_dev  element-major [F][E][N], node-major [F][N][E] (d in place of f); must not
 *            overlap the inputs
 * Errors: as lc_contract; LC_ERR_UNSUPPORTED when the kernel is not of this form (and
 * lc_contract returns it for kernels of this form).
 */
lc_status lc_contract_geo(const lc_kernel *k, const lc_variant *v, const void *D_dev, const void *u_dev,
                          const void *r_dev, void *out_dev, int64_t E, int32_t N, int32_t F, void *stream);

/*
 * The surface part of the dG operator (the dG FEM surface workload of Table 1): at each face
 * node the jump between the interior and the exterior trace, scaled per face, lifted to the
 * volume nodes by the lift matrix:
 *
 *     out[e, i] (+)= sum_{f,p} L[i, f, p] * s[e, f] * (u[e, fmask[f, p]] - u_flat[vmapP[e, f, p]])
 *
 * stated to lc_kernel_create as the domain { [e,i,f,p] : 0<=e<E and 0<=i<N and 0<=f<Nf and
 * 0<=p<Nfp } and, in exactly this form (names free), the instruction
 * "out[e,i] = sum((f,p), L[i,f,p]*s[e,f]*(u[e,fmask[f,p]] - u[vmapP[e,f,p]]))" (u read as a
 * flat array through vmapP).  FP32 SIMT engine (the contraction over f, p is short: about 5
 * flops per byte moved), element-major.
 *   L_dev      [N][Nf*Nfp] float          fmask_dev  [Nf*Nfp] int32, each in [0, N)
 *   vmapP_dev  [E][Nf*Nfp] int32, each in [0, E*N) (the element's own node on boundary faces)
 *   s_dev      [E][Nf] float               u_dev, out_dev  [E][N] float, out not overlapping
 *   accumulate 1: out += the lifted fluxes; 0: out = them
 * Sizes: 1 <= N <= 128, Nf * Nfp <= 256, E * N < 2^31.  Descriptor: engine SIMT, FP32,
 * element-major; prefetch_smem 1 (add_prefetch) has the bulk-copy engine stage, `stages`
 * (1 or 2) tiles ahead in as many buffers, each 64-element tile's vmapP rows, face scales,
 * u rows and up to 64 u rows on either side (fewer where shared memory is short) in shared
 * memory; exterior traces inside that window are read from there, the others from global
 * memory (u, vmapP and s must then be 16-byte aligned, else every operand is read from
 * global memory, as with prefetch_smem 0); ctas_per_sm (0 = 4) and max_ctas size the
 * persistent grid, which never exceeds the CTAs resident at once; tile_e 64 or 128 elements
 * per tile.  An index out
 * of range is not followed: its flux becomes NaN and lc_device_error reports LC_ERR_INDEX.
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_INVALID_VARIANT, LC_ERR_MISALIGNED (4-byte),
 * LC_ERR_NO_DEVICE, LC_ERR_UNSUPPORTED (not a kernel of this form), LC_ERR_CUDA.
 */
lc_status lc_lift(const lc_kernel *k, const lc_variant *v, const float *L_dev, const int32_t *fmask_dev,
                  const int32_t *vmapP_dev, const float *s_dev, const float *u_dev, float *out_dev, int64_t E,
                  int32_t N, int32_t Nf, int32_t Nfp, int32_t accumulate, void *stream);

/*
 * The contraction on host arrays: copies D and u from host to the caller's device
 * buffers, contracts, and copies out back to the host.  Large batches are cut into up to
 * 8 element chunks (whole tiles, >= 2^16 elements each) whose copies in, contractions
 * and copies out overlap: the copies run on two library-owned streams (one per
 * direction and device, created on first use and kept until exit), the contractions on `stream`,
 * ordered by events; all of it starts after the work already queued on `stream`, and
 * `stream` resumes after the last copy out.  Asynchronous with respect to the host when
 * the host buffers are page-locked; synchronise `stream` before reading out_host.  Not
 * for use inside a stream capture.  Calls on one device share the two copy streams: calls
 * from several threads stay correct, their copies take turns.
 *   D_host, u_host, out_host   host arrays with the layouts of lc_contract
 *   D_dev, u_dev, out_dev      device scratch of the same sizes (caller-owned); each chunk
 *                              packs its u and out at its element offset, so after the
 *                              call u_dev and out_dev hold chunk-packed data, not the
 *                              lc_contract layout (the same as it when there is one chunk)
 * Errors: as lc_contract, plus LC_ERR_CUDA for a failed copy.
 */
lc_status lc_contract_host(const lc_kernel *k, const lc_variant *v, const void *D_host,
                           const void *u_host, void *out_host, int64_t E, int32_t N, int32_t F,
                           void *D_dev, void *u_dev, void *out_dev, void *stream);

/*
 * Device error word: returns LC_ERR_TIMEOUT if any kernel recorded a bounded
 * wait that gave up since the last clear, else LC_ERR_INDEX if a kernel met an index out
 * of range (lc_lift), else LC_OK.  Synchronises the device.  clear != 0 resets the word.
 */
lc_status lc_device_error(int clear);

/*
 * Failure-path self-test: enqueue a one-warp kernel whose bounded mbarrier wait is made
 * to run out (nothing ever arrives) after limit_ns (1 ns .. 1 s).  The kernel then sets
 * the device error word exactly as a pipeline wait that gave up would, and returns; no
 * fault, no hang.  lc_device_error(…) then reports LC_ERR_TIMEOUT.
 */
lc_status lc_selftest_wait_timeout(int64_t limit_ns, void *stream);

/* ------------------------------------------------------------------------- */
/* Grouped launch: several problems of different sizes in one persistent      */
/* kernel, optionally captured once in a CUDA graph and replayed.             */
/* ------------------------------------------------------------------------- */
typedef struct lc_group {
    int64_t E;            /* elements of this group (>= 0) */
    int32_t N;            /* nodes, 1..256 */
    int32_t F;            /* operators, 1..8 */
    const void *D_dev;    /* [F][N][N] float */
    const void *u_dev;    /* layout per the variant */
    void *out_dev;        /* layout per the variant */
} lc_group;

typedef struct lc_grouped_plan lc_grouped_plan;

/* Workspace bytes lc_grouped_plan_create needs for these groups and variant. */
lc_status lc_grouped_workspace_size(const lc_kernel *k, const lc_variant *v, const lc_group *groups,
                                    int32_t ngroups, size_t *bytes);

/*
 * Plan one persistent launch over all groups.
 * FP32 SIMT variant: every group gets a SIMT tile shape with the same CTA size; all
 * (group, tile) work is cut into one contiguous range per CTA, balanced by estimated
 * cost.  The variant gives the register block (elems_per_thread, split_i), unroll (1 or
 * 4), prefetch_smem, stages and ctas_per_sm.
 * Tensor-core variant (TCGEN05, BF16 or BF16X3, at most 16 groups): each group that has
 * a tensor-core plan (lc_variant_validate's rules; the epilogue works in 8-column chunks)
 * for the variant, or else for the first of its changes "stages = 1", "the other K-block
 * width (elems_per_thread 1 <-> 64)", "store_rows = 32" (element-major) and their
 * combinations, with the same CTA size (unroll), runs in one tensor-core launch, one CTA per SM at most: every (group,
 * column block) unit gets at least one CTA, and the rest go to the unit whose estimated
 * time (tiles x per-tile cost / CTAs) is the largest.  More units than SMs is
 * LC_ERR_INVALID_VARIANT.  Groups without a tensor-core plan (e.g. N above the plans'
 * limit) run after it, each in a K-split FP32 launch (tiles of 128 elements, j chunks of 8,
 * one u buffer), or, without a K-split plan, in a FP32 SIMT grouped launch (8 x 8 register
 * blocks, unroll 4, two stages, three CTAs per SM); their results are FP32's, below both
 * reduced-precision bounds.
 *   workspace_dev  caller-owned device memory holding the group and work tables
 *                  (lc_grouped_workspace_size bytes, 16-byte aligned); it must outlive
 *                  the plan, as must the groups' buffers, which the plan references.
 *   use_graph      1: capture the launch on `stream` (not the legacy default stream)
 *                  into a CUDA graph; lc_grouped_run then replays it.
 * The tables are uploaded synchronously on `stream`.  The plan is a host object;
 * free it with lc_grouped_plan_destroy.
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_INVALID_VARIANT, LC_ERR_ASSUMPTION,
 * LC_ERR_MISALIGNED, LC_ERR_BUFFER_TOO_SMALL, LC_ERR_NO_DEVICE, LC_ERR_CUDA.
 */
lc_status lc_grouped_plan_create(const lc_kernel *k, const lc_variant *v, const lc_group *groups,
                                 int32_t ngroups, void *workspace_dev, size_t workspace_bytes,
                                 int32_t use_graph, void *stream, lc_grouped_plan **plan);

/* Enqueue the planned launch (graph replay when captured) on `stream`. */
lc_status lc_grouped_run(lc_grouped_plan *plan, void *stream);

/* Grid size (both launches) and number of (group, tile-range) segments of a plan (a
 * tensor-core CTA counts as one segment). */
lc_status lc_grouped_plan_info(const lc_grouped_plan *plan, int32_t *grid, int32_t *segments);

/*
 * The descriptor that serves group `group` (0-based, < ngroups) of a plan: the variant as
 * given (SIMT plans; tensor-core groups that have a plan for it), the tensor-core variant
 * the planner fell back to for that group, or the FP32 SIMT descriptor of the groups
 * without a tensor-core plan.  Errors: LC_ERR_INVALID_ARGUMENT.
 */
lc_status lc_grouped_plan_group(const lc_grouped_plan *plan, int32_t group, lc_variant *v);

void lc_grouped_plan_destroy(lc_grouped_plan *plan);

/* ------------------------------------------------------------------------- */
/* FP64 error norm on the GPU.                                               */
/* ------------------------------------------------------------------------- */
enum { LC_DTYPE_F32 = 0, LC_DTYPE_F64 = 1 };

/* Workspace bytes needed by lc_error_norm for n elements. */
lc_status lc_error_norm_workspace_size(int64_t n, size_t *bytes);

/*
 * sums_dev[0] = sum_k (out[k] - ref[k])^2,  sums_dev[1] = sum_k ref[k]^2, in FP64,
 * so that ||out - ref||_F / ||ref||_F = sqrt(sums[0] / sums[1]).  Deterministic:
 * fixed grid, per-block partial sums in `workspace_dev`, one final block.
 *   out_dev        n values of type out_dtype (LC_DTYPE_F32 or LC_DTYPE_F64)
 *   ref_dev        n doubles
 *   sums_dev       2 doubles (device)
 *   workspace_dev  lc_error_norm_workspace_size bytes, 16-byte aligned
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_BUFFER_TOO_SMALL, LC_ERR_MISALIGNED, LC_ERR_CUDA.
 */
lc_status lc_error_norm(const void *out_dev, int32_t out_dtype, const double *ref_dev,
                        int64_t n, double *sums_dev, void *workspace_dev,
                        size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------- */
/* Variant selection: exhaustive autotuning and the learned cost model.       */
/* The paper lets the controlling program choose transformations per target   */
/* and workload (Section 1); these calls make that choice measurable.         */
/* ------------------------------------------------------------------------- */

/*
 * The candidate descriptors for a problem (the autotuner's search space), valid ones
 * only, in a fixed order; descriptors whose plan (lc_variant_plan) has fewer than two
 * warps per CTA are left out (they remain valid for lc_contract).  Writes min(count, cap) entries; *count = the number of
 * candidates.  Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_BUFFER_TOO_SMALL (cap < count).
 */
lc_status lc_enumerate_variants(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout,
                                int32_t precision, lc_variant *out, int32_t cap, int32_t *count);

/*
 * Time every candidate on the caller's problem buffers (D, u, out as for lc_contract):
 * one warm-up launch, then the median of `reps` launches timed with CUDA events on
 * `stream`.  Synchronises the stream.  On return variants[0..count) and ms[0..count)
 * hold the candidates sorted by time, fastest first.  `out` is overwritten.
 * Errors: as lc_enumerate_variants and lc_contract.
 */
lc_status lc_autotune(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t precision,
                      const void *D_dev, const void *u_dev, void *out_dev, int32_t reps, lc_variant *variants,
                      float *ms, int32_t cap, int32_t *count, void *stream);

/*
 * MLP cost model: inputs x[din] (1 <= din <= 32), three hidden ReLU layers of width
 * 64, one linear output (the predicted log run time).  Parameters are one float
 * vector, in this order: W1[64][din], b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
 * w4[64], b4[1]; all pointers below are device pointers, arrays row-major.
 */
lc_status lc_mlp_param_count(int32_t din, int64_t *count);

/* y[s] = network(X[s][0..din)) for s < n. */
lc_status lc_mlp_forward(const float *params_dev, const float *X_dev, int64_t n, int32_t din, float *y_dev,
                         void *stream);

/* Workspace bytes for lc_mlp_loss_grad. */
lc_status lc_mlp_workspace_size(int32_t din, size_t *bytes);

/*
 * Mean squared error L = (1/n) sum_s (y_s - t_s)^2 and its gradient by backpropagation:
 * grad_loss_dev[0..P) = dL/dparams, grad_loss_dev[P] = L (P = lc_mlp_param_count).
 * Deterministic (fixed per-block partial sums, then an ordered reduction).
 */
lc_status lc_mlp_loss_grad(const float *params_dev, const float *X_dev, const float *t_dev, int64_t n,
                           int32_t din, float *grad_loss_dev, void *workspace_dev, size_t workspace_bytes,
                           void *stream);

/* One Adam update (bias-corrected, step >= 1) of n parameters with moments m, v. */
lc_status lc_mlp_adam_step(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int64_t n,
                           int32_t step, float lr, float beta1, float beta2, float eps, void *stream);

/*
 * The learned pick (Section 1: the controlling program chooses the transformations per
 * target and workload).  The cost model reads LC_FEATURES features of a (problem,
 * descriptor) pair: problem size and requested path, the descriptor's fields, and the
 * launch plan lc_variant_plan resolves it to (grid, tiles per CTA, column blocks, shared
 * memory, threads, tensor-core instructions per CTA, ...); every feature is O(1).
 */
#define LC_FEATURES 32

/*
 * x[0..LC_FEATURES) = the features of descriptor v for the problem (E, N, F) stored in
 * `layout` and requested at `precision` (the path asked for; v->precision is the one it
 * runs).  Host only; uses the current device's SM count and shared memory when there is
 * one (else a 148-SM, 227 KB part).  Errors: those of lc_variant_plan.
 */
lc_status lc_variant_features(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout,
                              int32_t precision, const lc_variant *v, float *x);

/* Workspace bytes lc_pick_variant needs (room for the features and predictions of up to
 * 256 candidates). */
lc_status lc_pick_workspace_size(size_t *bytes);

/*
 * Pick a descriptor with a trained cost model: enumerate the candidates
 * (lc_enumerate_variants), build their features (lc_variant_features), predict their log
 * run time with lc_mlp_forward on `stream` (din = LC_FEATURES), and return the candidate
 * with the smallest prediction (the first one on ties) in *picked, its prediction in
 * *predicted (may be NULL).  Synchronises `stream`.
 *   params_dev     the network's parameters (lc_mlp_param_count(LC_FEATURES) floats)
 *   workspace_dev  lc_pick_workspace_size bytes, 16-byte aligned (features, predictions)
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_BUFFER_TOO_SMALL, LC_ERR_MISALIGNED,
 * LC_ERR_UNSUPPORTED (no candidate for this problem), LC_ERR_CUDA.
 */
lc_status lc_pick_variant(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout, int32_t precision,
                          const float *params_dev, void *workspace_dev, size_t workspace_bytes,
                          lc_variant *picked, float *predicted, void *stream);

/*
 * lc_pick_variant with an ensemble of n_models networks of the same shape, trained apart
 * (different initialisations and minibatch orders): each candidate's prediction is the mean
 * of the models' predicted log run times (models taken in order), and the candidate with
 * the smallest mean is returned (*predicted = that mean).  Averaging removes much of one
 * network's variance between trainings (held-out regret of single networks differs by
 * several points from seed to seed).  lc_pick_variant is the case n_models = 1.
 *   params_dev  n_models consecutive parameter blocks of lc_mlp_param_count(LC_FEATURES)
 *               floats each, 4-byte aligned
 *   n_models    1 to 64
 * Errors: those of lc_pick_variant.
 */
lc_status lc_pick_variant_ensemble(const lc_kernel *k, int64_t E, int32_t N, int32_t F, int32_t layout,
                                   int32_t precision, const float *params_dev, int32_t n_models,
                                   void *workspace_dev, size_t workspace_bytes, lc_variant *picked,
                                   float *predicted, void *stream);

/*
 * lc_error_norm without a workspace, for callers that cannot allocate device memory
 * (cudaMalloc synchronises the device, which latency-bound or real-time callers forbid,
 * and some host frameworks give their plugins no allocator).  This call has no
 * counterpart in the paper; it exists only for such callers.
 *   out_dev, ref_dev, sums_dev   as for lc_error_norm; 1 <= n <= 2^28
 * The partial sums live in a 64 KiB array in device memory that the library holds on
 * every GPU it is loaded on until the process exits; nothing is allocated per call.
 * The grid (at most 4096 blocks of 256 threads, one per 1024 elements) grid-strides
 * through larger inputs.
 * The array's address is looked up on the first call made on each device (with that
 * device current); make that first call before any stream capture.  All calls share the
 * array, so calls that overlap on the GPU race: serialise them.  Each call rewrites the
 * slots it uses, so no clearing is needed.  Results equal lc_error_norm's up to the
 * order of the FP64 summation.
 * Errors: LC_ERR_INVALID_ARGUMENT, LC_ERR_BUFFER_TOO_SMALL (n above 2^28, the array's
 * capacity), LC_ERR_MISALIGNED, LC_ERR_CUDA.
 */
lc_status lc_error_norm_noalloc(const void *out_dev, int32_t out_dtype, const double *ref_dev, int64_t n,
                                double *sums_dev, void *stream);

/* Number of SMs and compute capability of the current device. */
lc_status lc_device_info(int32_t *sm_count, int32_t *cc_major, int32_t *cc_minor);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
