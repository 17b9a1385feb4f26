// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lc.h"

namespace lc {

// Parsed kernel: loop domain + one contraction instruction + assumptions (Section 2.1).
struct Assumption {
    std::string param;  // parameter name
    int op;             // 0: mod k = 0, 1: >=, 2: >, 3: <=, 4: <, 5: =
    long long k;
};

// What the instruction computes (each kind has its own entry point).
enum KernelKind { KIND_CONTRACT = 0, KIND_GEO = 1, KIND_ELEMENTWISE = 2, KIND_LIFT = 3 };

// Elementwise instruction: an expression tree over array loads, scalar parameters and
// constants.  arrays[0] is the output; the inputs follow in order of first appearance.
enum EwOp { EW_LOAD, EW_PARAM, EW_CONST, EW_ADD, EW_SUB, EW_MUL, EW_DIV, EW_NEG };
struct EwNode {
    int op;
    int a = -1, b = -1;  // operands (node indices)
    int arg = -1;        // EW_LOAD: array index; EW_PARAM: parameter index
    double val = 0.0;    // EW_CONST
};
struct EwArray {
    std::string name;
    std::vector<int> dims;  // domain positions of its indices, ascending
};
struct Elementwise {
    std::vector<EwNode> nodes;
    int root = -1;
    std::vector<EwArray> arrays;
    std::vector<std::string> params;
};

struct Kernel {
    int kind = KIND_CONTRACT;
    std::string g_name, d_iname;      // KIND_GEO: geometric-factor array G[e,d,f], physical-derivative iname
    Elementwise ew;                   // KIND_ELEMENTWISE
    std::string s_name, fmask_name, vmap_name, p_iname, Nf_param, Nfp_param;  // KIND_LIFT
    std::vector<std::string> inames;  // as written in the domain
    std::vector<std::string> bounds;  // parameter bounding each iname
    std::string out_name, d_name, u_name;
    std::string f_iname, e_iname, i_iname, j_iname;  // roles ("" for f in the F = 1 form)
    std::string F_param, E_param, N_param;           // "" for F in the F = 1 form
    std::vector<Assumption> assumptions;
    std::string domain_text, insn_text, assumptions_text;
};

// Launch geometry resolved from a descriptor and a problem size.
struct SimtGeom {
    int VEC;       // elements per 16-byte vector
    int RE, RC;    // register block: elements x columns per thread
    int EG, CG;    // thread grid: element groups x column groups
    int WC;        // lanes of a warp along columns (the warp is (32 / WC) x WC)
    int stages;    // u tiles in flight (prefetch ring depth)
    int bulk;      // u tiles fetched by the bulk-copy engine
    int bulk_store;  // element-major output tiles written by bulk stores
    int TE;        // elements per tile (= EG * RE)
    int CW;        // columns of the resident D^T block (= CG * RC >= G * N)
    int G;         // operators per column block (one block per CTA)
    int isplit;    // > 0: blocks are row ranges of one operator (its D^T does not fit)
    int nchunks;   // column blocks: ceil(F / G)
    int threads;   // EG * CG
    size_t smem;   // dynamic shared memory bytes
    long long ntiles;
    int grid;
};

struct SimtArgs {
    const void *D;
    const void *u;
    void *out;
    long long E;
    int N, F, C;
    int TE, EG, CG, CW, nchunks;
    int G;          // operators per column block
    int isplit;     // > 0: column blocks are row ranges of this many rows of one operator
    int WC, stages, bulk, bulk_store;
    long long ntiles;
    int tail_free;
    unsigned int *err;
};

// Warp-per-element-group kernel for small N.
struct WarpArgs {
    const void *D;
    const void *u;
    void *out;
    long long E;
    int N, F;
    int per_warp;     // elements handled by one warp per step (32 / N rounded down)
    long long ngroups;
    int tail_free;
};

// K-split SIMT kernel (FP32): 8 x 8 register blocks over a BM x 128 output tile, the
// reduction over j cut into chunks of BK (split_iname on j) whose D^T slices are fetched
// asynchronously into a two-slot ring, the u tile resident (transposed) for all column blocks.
struct KsArgs {
    const float *D;
    const float *u;
    float *out;
    long long E;
    int N, F, C;       // C = F * N output columns
    int Kp, nkc;       // N rounded up to the chunk width, and the number of chunks
    int nblocks;       // column blocks of 128
    long long ntiles;  // element tiles of BM
    int ubufs;         // u tile buffers: 2 = the next tile's u is fetched during this tile
    int vec_u;         // node-major: 16-byte copies of u rows (E % 4 == 0)
    int vec_out;       // 16-byte output stores (element-major: N % 4 == 0; node-major: E % 4 == 0)
};
// set_attr: set the instance's shared-memory size first; grid <= 0: only that.
lc_status ks_launch(const KsArgs &a, int layout, int bm, int bk, int grid, cudaStream_t s, bool set_attr = true);
size_t ks_smem_bytes(int Kp, int bm, int bk, int ubufs);

// Tensor-core kernel (tcgen05): one column block of G operators per CTA.
struct TcArgs {
    const float *D;
    const float *u;
    float *out;
    const float *r;  // volume derivative: per-element geometric factors (null for the contraction)
    long long E;
    int N, F;
    int G;          // operators per column block
    int nblocks;    // column blocks (ceil(F / G))
    int Np;         // accumulator columns per operator: N rounded up to 16 (or to 8)
    int chunk;      // epilogue chunk: 16 columns when Np is a multiple of 16, else 8
    int CB, CBp;    // columns per block (G * Np) and the MMA N (CB rounded up to 16)
    int Kp, KB, nkb;  // K padded to the block width, K-block width (16/32/64 -> 32/64/128-byte swizzle), blocks
    int Kt;         // K the MMAs read: N rounded up to 16 (zeros past N)
    int stack;      // BF16X3 with two B terms stacked along N (2 * CBp <= 256): 5 MMAs per K step, not 6
    int tmem_cols;  // columns per accumulator (power of two >= CBp, or >= 2 * CBp when stacked)
    int a_tmem;     // 1: the A terms live in tensor memory after the two accumulators
    int a_cols;     // tensor-memory columns per A buffer (NT terms x K/2 packed bf16 pairs)
    int tmem_alloc; // tensor-memory columns allocated (power of two >= 32)
    int stages;     // u stage buffers (1 to 3)
    int early_release;  // 1: conversion threads take their chunks into registers, then free the stage
    int threads_per_row;       // epilogue threads per tile row
    int conv_threads_per_row;  // conversion threads per tile row (CTA = 128 * (both) + 64 threads)
    int abufs;      // A-operand buffers (1 or 2)
    int obufs;      // element-major output staging slots of one operator-tile (1 to 4)
    int store_quarters;  // element-major: TMEM lane quarters (32 rows each) per bulk store: 1, 2 or 4
    int store_warp;      // 1: whole-tile element-major slots are written out by the CTA's store warp
    long long ntiles;
    int bulk_u, bulk_store;
    unsigned int *err;
    unsigned int off_stage, off_out, off_bar, smem_bytes;
};

lc_status tc_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s);

// Threads of a tensor-core CTA: 4 x (epilogue + conversion threads per tile row) warps, then
// the producer, MMA and store warps.
static inline int tc_threads(const TcArgs &a) { return 128 * (a.threads_per_row + a.conv_threads_per_row) + 96; }

// Grouped tensor-core launch: per-group plans and the per-CTA unit table.
static constexpr int kTcMaxGroups = 16;
struct TcGroupedParams {
    TcArgs g[kTcMaxGroups];
    const int4 *map;  // per CTA: {group, column block, first tile, tile step} (device memory)
    int ngroups;
};
lc_status tc_grouped_launch(const TcGroupedParams &P, int layout, int nterms, int grid, int threads, size_t smem,
                            cudaStream_t s, void **fn_out);

// Surface lift of the dG operator (lift.cu).
struct LiftArgs {
    const float *L;        // [N][M] lift matrix
    const int *fmask;      // [M] element node of face node m
    const int *vmapP;      // [E][M] exterior trace: index into u as a flat array
    const float *s;        // [E][Nf] per-face scale
    const float *u;        // [E][N]
    float *out;            // [E][N]
    long long E;
    int N, Nf, Nfp, M;
    int accumulate;
    int halo;              // >= 0: the tile's vmapP rows, scales, u rows and `halo` u rows on
                           // either side are staged in shared memory (bulk copies, nbuf tiles
                           // ahead) and exterior traces inside that window read from there;
                           // -1: every operand read from global memory
    int nbuf;              // staging buffers (1 or 2)
    int te;                // elements per tile (64 or 128)
    unsigned int *err;     // device error word: bit 1 set on an index out of range
};
lc_status lift_launch(const LiftArgs &a, int grid, cudaStream_t s);
size_t lift_smem_bytes(int N, int M, int Nf, int halo, int nbuf, int te);
int lift_threads(int N, int te);

// Elementwise kernels: check a descriptor against extents (one per iname) without launching;
// reports the grid and the number of tiles.
lc_status ew_validate(const Kernel &K, const lc_variant *v, const int64_t *extents, bool need_device, int *grid,
                      long long *ntiles);
lc_status tc_geo_launch(const TcArgs &a, int layout, int nterms, int grid, cudaStream_t s);

// Grouped launch: per-group SIMT arguments, contiguous tile ranges, ranges per CTA.
struct GroupSeg {
    int group;
    int chunk;  // column block of the group
    long long first, count, step;  // tiles first, first + step, ... (count of them)
};
struct GroupedArgs {
    const SimtArgs *groups;
    const GroupSeg *segs;
    const int *cta_seg;  // CTA b walks segs[cta_seg[b] .. cta_seg[b+1])
    unsigned int *err;
};
void *grouped_kernel_ptr(int layout, int re, int rc, int unr, int pf);

int sm_count();
int current_cc(int *major, int *minor);
unsigned int *error_word();
lc_status cuda_fail(cudaError_t e);
size_t smem_optin_limit();

// SIMT launchers (one per element type / layout translation unit).
lc_status simt_launch_f32_elem(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s);
lc_status simt_launch_f32_node(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s);
lc_status simt_launch_f64_elem(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s);
lc_status simt_launch_f64_node(const SimtArgs &a, const SimtGeom &g, int unroll, int prefetch,
                               cudaStream_t s);
lc_status warp_launch(const WarpArgs &a, int layout, int fp64, int grid, int threads, cudaStream_t s);

}  // namespace lc

// The opaque handle of the C ABI: an immutable parsed kernel.
struct lc_kernel {
    lc::Kernel k;
};

