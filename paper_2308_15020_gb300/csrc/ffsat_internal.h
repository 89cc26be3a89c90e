// Internal data layout shared by the host code (ffsat_api.cpp) and the kernels.
// Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

struct ffsat_instance;

namespace ffsat {

// Literals per lane on the product (closed-form) path.
constexpr int kProdR = 8;
// Largest number of clauses per lane in one clause task (groups of 32 clauses;
// the host picks 1, 2 or 4 per instance and kernel width).
constexpr int kClausePerLane = 4;
// Packed literal: (variable << 1) | negated.  Padding literal: -1.
constexpr int32_t kPadLit = -1;

// Warp tasks.  task.x = kind | (G << 8) where G = lanes per constraint segment
// (power of two, 1..32); task.y = first item; task.z = item count; task.w = node
// count J of the largest constraint in the task (node path only).
// TASK_XOR2: records of XOR constraints of <= 2 literals in the clause array
// (two literals and the dummy, in any order, the dummy negated for even parity;
// FP32 weight bits last), same layout and grouping as TASK_CLAUSE.
enum : int32_t { TASK_CLAUSE = 0, TASK_PROD = 1, TASK_NODE = 2, TASK_XOR2 = 3 };

// Closed-form product constraints: FE = c0 + c1 prod_i (a + b y_i).
enum : int32_t { PROD_OR = 0, PROD_XOR_EVEN = 1, PROD_XOR_ODD = 2 };

// Where the fused kernel keeps a point's x and gradient accumulator, and the
// instance's constraint data (SMEM_RES: all three in shared memory; in FP32 the
// accumulator is then two int32 words per variable, see fix_s1).
enum : int32_t { SMEM_FULL = 0, SMEM_X = 1, SMEM_NONE = 2, SMEM_RES = 3 };

// Node task of an instance: the imaginary-node form (stable form) or the
// generic alpha + beta y factors (paper form).
enum : int32_t { NODE_FORM_IMAG = 0, NODE_FORM_GENERIC = 1 };

// Makes a device current for the lifetime of the guard and restores the
// caller's current device when it ends, so that no entry point leaves the
// calling thread on another device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t set(int device) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) {
            prev = -1;
            return e;
        }
        return prev == device ? cudaSuccess : cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Device status bits.
enum : int32_t { STATUS_NAN = 1, STATUS_OTHER = 2 };

// Everything a kernel reads, passed by value.
struct DevView {
    int32_t n;
    int32_t m;
    int32_t n_task;
    int32_t n_seg;
    const int4 *tasks;
    // thread-per-clause path (clauses of <= 3 literals)
    int32_t n_clause;
    int32_t pad0;
    const int4 *clauses;      // {l0, l1, l2, float bits of the FP32 weight}
    const double *clause_wd;  // FP64 weights
    // segment path (product and node constraints), sorted by length, descending:
    // segmeta[s] = {offset into seg_lits, length, aux, float bits of the FP32 weight};
    // aux = node-table offset (in nodes) on the node path, PROD_* kind on the product path
    const int4 *segmeta;
    const double *seg_wd;
    const int32_t *seg_lits;  // packed literals
    // Resident image {tasks | clauses | segmeta | seg_lits} (int4 units); tasks,
    // clauses, segmeta and seg_lits above point into it.  When it fits in shared
    // memory beside x and g, the kernel copies it there once per CTA.
    const int4 *res_image;
    int32_t res_int4, res_off_tasks, res_off_clauses, res_off_segmeta, res_off_lits, pad1;
    // node tables of the generic node task (paper form) and of the plain FP64
    // comparator, 8 reals per node: alpha.re, alpha.im, beta.re, beta.im, d.re,
    // d.im, c.re, c.im
    const float4 *tab_f;
    const double *tab_d;
    // node tables of the imaginary-node form (stable form), 4 words per node:
    // FP32 {t, C.re, C.im, ec (int bits)}, FP64 {t, C.re, C.im, ec}; the C
    // mantissa has its largest component in [1/2, 1) and is scaled by 2^ec;
    // entry 0 is an all-zero node
    const float4 *tab_im_f;
    const double *tab_im_d;
    int32_t node_form;  // NODE_FORM_IMAG or NODE_FORM_GENERIC: which node task runs
    int32_t fix_two;    // the FP32 fixed-point gradient uses its lo word too (else hi alone)
    // device constants of f under the current weights: [0] = sum over clauses of
    // -w plus sum of w FE over constant constraints (fused kernel), [1] = the
    // latter alone (plain FP64 path); rewritten on the device by the ERWA update
    const double *f_const;
    // Two-word fixed-point gradient accumulator of the FP32 shared-resident mode:
    // g = hi / 2^S1 + lo / 2^(S1+S2); fix_s1 = 2^S1, fix_s2 = 2^S2 and the inverses.
    float fix_s1, fix_s2, fix_i1, fix_i12;
    // fixed-point gradient of the FP64 cluster step, two 32-bit words per
    // variable: g = (hi 2^L + lo) / 2^S64; fix64_s = 2^S64, fix64_i = 2^-S64,
    // fix64_l = L
    double fix64_s, fix64_i;
    int32_t fix64_l;
    int32_t has_prod;  // the image has product-path segments (FP64: FP64 product words in use)
    // start value of both fixed-point words of variable v (npad entries):
    // -(fixed-point contributions v receives per evaluation) * 0x4B400000 mod 2^32
    const int32_t *fix_bias;
    // exact-check CSR over all constraints (packed literals)
    const int32_t *row_ptr;
    const int32_t *lits;
    const uint8_t *type;
    const int32_t *param;
    // plain FP64 comparator
    const int32_t *cons_tab;  // node-table offset, or -1 for closed forms
    const double *cons_wd;
    int32_t *status;
};

struct StepParams {
    int32_t T;
    int32_t restart;
    double lr;
    uint64_t seed, epoch, b_offset;
};

// Threads per CTA of the fused kernel for (real type, node R).
constexpr int fused_threads(bool f64, int node_r) {
    return f64 ? (node_r >= 16 ? 128 : 256) : (node_r >= 16 ? 512 : (node_r > 0 ? 512 : 1024));
}

// Threads per CTA of the batch kernel: as the fused kernel; FP32 node-path
// batches also have a 384-thread instance (ffsat_batch_create may pick it).
constexpr int batch_threads_default(bool f64, int node_r) { return fused_threads(f64, node_r); }

// Mode of the fused kernel.
enum : int32_t { MODE_EVAL = 0, MODE_STEP = 1, MODE_PGFP = 2 };

struct FusedArgs {
    int32_t B;
    int32_t mode;
    const void *x_in;
    void *x_out;
    double *f;
    void *g;          // eval: output rows (may be NULL)
    void *g_scratch;  // step with g outside shared memory: [B, n] accumulator
    StepParams sp;
    uint8_t *solved;
    int32_t *n_unsat;
    int32_t *unsat_counts;  // step: per-constraint violation counts added by the final check (may be NULL)
    // MODE_PGFP (line-search step; sp.lr is the initial step size): backtracking
    // factor, trials per iteration, smallest step, absolute slack of the
    // sufficient-decrease test, [B, n] scratch for the extrapolated points, and
    // optional per-point outputs (iterations taken, final step size)
    double beta, eta_min, slack;
    int32_t maxls;
    int32_t pairs;  // MODE_STEP: two points per CTA (FP32 resident image, one fixed-point word)
    void *y_scratch;
    int32_t *iters;
    double *eta_out;
};

// One instance of a batch launch.
struct BatchInst {
    DevView V;
    FusedArgs A;
    int32_t mode;  // shared-memory mode of the instance for the launch's real type
    int32_t pad[3];
};

// Batch-kernel launchers (f64: real type; node_r: 0 or 16; threads: the CTA
// width, 384 or 512 for FP32 with node_r 16, ignored otherwise).  With
// prepare_only the launcher raises the dynamic shared-memory limit to `smem` and
// reports through *blocks_per_sm how many CTAs of the kernel fit on one SM.
cudaError_t launch_batch(bool f64, int node_r, int threads, const BatchInst *insts, const int2 *items, int n_items,
                         int *counter, const StepParams &sp, size_t smem, int grid, cudaStream_t s, bool prepare_only,
                         int *blocks_per_sm);
#define FFSAT_BATCH_LAUNCHER(name)                                                                       \
    cudaError_t name(const BatchInst *insts, const int2 *items, int n_items, int *counter, const StepParams &sp, \
                     size_t smem, int grid, cudaStream_t s, bool prepare_only, int *blocks_per_sm)
FFSAT_BATCH_LAUNCHER(batch_f32_r16_t384);
FFSAT_BATCH_LAUNCHER(batch_f32_r16_t512);
FFSAT_BATCH_LAUNCHER(batch_f32_r0);
FFSAT_BATCH_LAUNCHER(batch_f64_r16);
FFSAT_BATCH_LAUNCHER(batch_f64_r0);

// Fused-kernel launchers, one per (real type, node R); each handles the three
// shared-memory modes.  With prepare_only the launcher only raises the kernel's
// dynamic shared-memory limit to `smem`.
#define FFSAT_FUSED_LAUNCHER(name)                                                                   \
    cudaError_t name(const DevView &V, int smem_mode, const FusedArgs &a, size_t smem, int grid, \
                     cudaStream_t s, bool prepare_only)
FFSAT_FUSED_LAUNCHER(fused_f32_r0);
FFSAT_FUSED_LAUNCHER(fused_f32_r8);
FFSAT_FUSED_LAUNCHER(fused_f32_r16);
FFSAT_FUSED_LAUNCHER(fused_f64_r0);
FFSAT_FUSED_LAUNCHER(fused_f64_r8);
FFSAT_FUSED_LAUNCHER(fused_f64_r16);

// Device address of the statically reserved scratch (FFSAT_STATIC_SCRATCH_BYTES)
// on `device`, which must be current; looked up on the first call per device.
cudaError_t static_scratch(int device, void **ptr);

// Graph view of an instance for the learned restart proposal (device arrays).
struct GraphView {
    int device;
    int n, m;
    const int32_t *row_ptr;   // constraint -> literals (CSR)
    const uint32_t *lits;     // variable | negated << 31
    const int32_t *var_ptr;   // variable -> occurrences (transposed CSR)
    const uint32_t *var_occ;  // constraint | negated << 31
    const float *fv;          // [n, 8] variable features
    const float *fc;          // [m, 8] constraint features
    const float *inv_deg;     // [n] 1 / occurrences (0 if none)
    const float *inv_len;     // [m] 1 / length
};

// Build the graph view on first use (host preprocessing + one upload), then
// return it.  Returns an ffsat status code.
int instance_graph(::ffsat_instance *inst, GraphView *out);
// Record an error message for ffsat_last_error(); returns code.
int set_error(int code, const char *msg);

// Exact checker: one CTA per point.
cudaError_t launch_check(const DevView &V, bool f64, int B, const void *x, uint8_t *sat, int32_t *n_unsat,
                         int32_t *U, cudaStream_t s);
// Plain FP64 comparator; *launches receives the number of kernels enqueued.
cudaError_t launch_plain64(const DevView &V, int B, const double *x, double *f, double *g, int32_t n_node,
                           const int32_t *node_ids, int32_t n_closed, const int32_t *closed_ids,
                           cudaStream_t s, int *launches);

}  // namespace ffsat
