// crk_internal.cuh -- engine context, device buffers and small device helpers
// shared by the CUDA translation units of the CRKSPH pair engine.
#pragma once

#include <cuda.h>   // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>

#include "crk.h"

namespace crk {

constexpr int TILE = 32;          // particles per tile = one warp
constexpr int MAX_LEVELS = 32;    // tile-tree levels (ntiles < 2^31)
constexpr float TWO_M32 = 2.3283064365386963e-10f;   // 2^-32
constexpr double PI_D = 3.14159265358979323846;

// device counters (unsigned long long slots in ctx->counters)
enum {
    CNT_GLIST = 0,      // gather-list entries allocated
    CNT_ULIST = 1,      // union-list entries allocated
    CNT_PAIRS_G = 2,    // gather pairs (excl. self) of the last P1
    CNT_PAIRS_U = 3,    // ordered union pairs of the last P4
    CNT_ERR_INPUT = 4,  // invalid particle records found
    CNT_HMAX = 5,       // max h as float bits
    CNT_WORK = 6,       // dynamic tile counter of the persistent pair kernels
    CNT_NOTDONE = 7,    // h iteration: particles not converged
    CNT_DTMIN = 8,      // min per-particle time step (float bits)
    CNT_ENTRIES = 9,    // stored-force units (32 entries) of the last list build
    CNT_MAXCNT = 10,    // largest pair-set count of the last walk
    CNT_MLP_ERR = 11,   // invalid records seen by the feature kernels
    CNT_GRAPH_ERR = 12, // sticky: some replayed step overflowed a capacity or saw invalid records
    CNT_TNEXT = 13,     // time bins: earliest step end over the leaves (ticks)
    CNT_CHANGED = 14,   // time bins: a limiter sweep raised some level
    CNT_UNRES = 15,     // time bins: particle level requests deeper than L
    CNT_WAKE = 16,      // time bins: passive leaves raised
    CNT_NACT = 17,      // time bins: leaves ending a step at the current tick (and 18: their particles)
    CNT_NEXT_OK = 19,   // du_next holds the next opening kick's energy rate for dt_next
    CNT_SKIP = 20,      // this step's opening kick takes du_next
    CNT_PO_MISS = 21,   // pair-once: tile pairs (I, J) whose reverse (J, I) was not found (sticky)
    CNT_WALK_TESTS = 22,  // lane tests of the exact predicate in the last list walk
    CNT_TMA_ERR = 23,   // sticky: a TMA-fed pass gave up waiting on its copies
    CNT_COUNT = 24
};

// Pass-input records in sorted order.
struct CorrRec {      // A, B, grad A, grad B of one particle (16 floats)
    float4 c0;        // A, Bx, By, Bz
    float4 c1;        // gAx, gAy, gAz, gB00
    float4 c2;        // gB01, gB02, gB10, gB11
    float4 c3;        // gB12, gB20, gB21, gB22
};
struct GvRec {        // grad v (9 floats) padded to 12
    float4 g0;        // g00 g01 g02 g10
    float4 g1;        // g11 g12 g20 g21
    float4 g2;        // g22 - - -
};

struct Buf {          // one device allocation
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace crk

struct crk_ctx {
    crk_params p;
    char err[512];
    int device = 0;
    int nsm = 0;

    // capacity of the per-particle buffers
    int cap_n = 0;
    int cap_tiles = 0;
    long long cap_glist = 0, cap_ulist = 0;

    // last build
    int n = 0;
    int ntiles = 0;
    int nlevels = 0;
    int level_off[crk::MAX_LEVELS];
    int level_cnt[crk::MAX_LEVELS];
    int built = 0;
    int cell_k = 0;
    long long glist_total = 0, ulist_total = 0;

    // sort scratch
    uint32_t *key_a = nullptr, *key_b = nullptr;
    int32_t *idx_a = nullptr, *idx_b = nullptr;
    uint32_t *hist = nullptr;        // 256 * nblocks (+ scan scratch)
    uint32_t *scan_tmp = nullptr;
    int cap_hist = 0;

    // sorted particle data
    uint4 *q4 = nullptr;             // (qx, qy, qz, H)
    float *hs = nullptr;             // h
    int32_t *perm = nullptr;         // sorted slot -> caller index
    uint32_t *keys = nullptr;        // sorted Morton keys

    // tiles and tree: all levels concatenated, level 0 = tiles
    uint4 *node_lo = nullptr;        // (xlo, ylo, zlo, Hmax)
    uint4 *node_hi = nullptr;        // (xhi, yhi, zhi, count)
    int cap_nodes = 0;

    // interaction lists: per tile (offset, count) and entries (tile ids)
    uint2 *gofs = nullptr, *uofs = nullptr;
    uint32_t *glist = nullptr, *ulist = nullptr;

    // chaining-mesh cell table (8^kmax + 1)
    int32_t *cell_start = nullptr;

    // device counters
    unsigned long long *counters = nullptr;
    unsigned long long *h_counters = nullptr;   // pinned host mirror

    // per-particle neighbour lists (column layout per tile) and stored pair forces
    uint4 *qV = nullptr;             // (qx, qy, qz, V bits)
    int32_t *cnt_g = nullptr, *cnt_u = nullptr;   // gather (j != i) and pair-set counts
    uint32_t *len_g = nullptr, *len_u = nullptr;  // per-tile max counts
    uint32_t *tcap = nullptr, *tbase = nullptr;   // per-tile stored-force base (units of 32)
    uint32_t *ent = nullptr;         // list entries: j | (j's kernel reaches i) << 31
    float4 *Fst = nullptr;           // F_ij per entry (P4 -> P5), compact layout
    int2 *lowc = nullptr;            // per particle: gather and other list entries with j < i
    int32_t *po_self = nullptr;      // pair-once: position of each tile in its own tile list
    uint32_t *po_rev = nullptr;      // pair-once: for tile-list entry (I, J), J >= I, the entry (J, I)
    uint2 *po_tofs = nullptr;        // pair-once: copy of the tile lists its P4 ran with (offset, count)
    uint32_t *po_tlist = nullptr;    //   and their entries
    float4 *po_rowA = nullptr;       // pair-once: j-side sums per (tile-list entry, lane): P4 (F, du)
    float2 *po_rowB = nullptr;       // P4 (Q, vsig); P5 (du, du of the second kick)
    long long po_cap = 0;            // tile-list entries the pair-once arrays hold
    int fst_po = 0;                  // Fst holds the pair-once form (owned entries only)
    long long ent_cap = 0, f_cap = 0, entries = 0;
    int kcap = 384;                  // list columns per particle
    int volumes_only = 0;            // walk without writing lists (no list buffer)
    int lists_valid = 0;
    float4 *frec = nullptr;          // packed pair-set records, 10 float4 (160 B) per particle
    CUtensorMap frec_map;            // TMA view of frec: rows of its first 36 floats (P4's TMA variant)
    const void *frec_map_base = nullptr;
    int frec_map_rows = -1;
    float *sfun = nullptr;           // specific entropy of the evaluation state
    float4 *sig = nullptr;           // (v + v') of a kick, s
    float4 *sig2 = nullptr;          // two kicks (closing, next opening): sig side by side, 2 per particle
    float *du_next = nullptr;        // the next step's opening-kick energy rate (formed ahead)
    double *dtb_next = nullptr;      // the next step's dt per box (batched; one box uses d_scalars[16])

    // pass buffers in sorted order
    float *V = nullptr, *Nn = nullptr;
    float4 *vel = nullptr;           // (vx, vy, vz, u) of the evaluation state
    float *mass = nullptr;
    crk::CorrRec *corr = nullptr;
    crk::GvRec *gv = nullptr;
    float4 *acc = nullptr;           // (ax, ay, az, dudt)
    float2 *vq = nullptr;            // (vsig, qmax)
    float4 *vb = nullptr, *va = nullptr;  // velocities before/after a kick (w unused)
    float *du = nullptr;

    // step state (sorted order)
    float4 *st_pos = nullptr;        // (x, y, z, h) positions of the state
    float4 *st_vel = nullptr;        // (vx, vy, vz, u) of the state
    float4 *st_half = nullptr;       // (p_1/2, u_1/2)
    float4 *st_tmp = nullptr;        // permutation scratch
    float *st_tmp1 = nullptr;
    uint4 *q_tmp = nullptr;          // build scratch: fixed-point records in input order
    float *h_tmp = nullptr;          // build scratch: h in input order
    int32_t *flags = nullptr;        // h iteration: converged flags
    double *d_red = nullptr;         // FP64 reduction scratch
    float *d_dt = nullptr;           // per-particle dt scratch
    float *rho = nullptr;            // RK-corrected density (crk_params.density = 1)
    double *d_scalars = nullptr;     // [0] dt of the step, [1] dt_next, [2..] diagnostics
    int rates_valid = 0;
    int step_n = 0;
    int h_iters = 0;                 // h_mode >= 1: P1 passes of the last step's eq:hi solve
    long long h_unconv = 0;          // particles it left unconverged

    // learned smoothing-length proposal (network state and feature grid)
    float *mlp_w = nullptr;          // FP32 master weights, CRK_MLP_NPARAM
    float *mlp_m = nullptr, *mlp_v = nullptr;   // Adam first and second moments
    float *mlp_part = nullptr;       // per-block gradient partials of one step
    int cap_part = 0;                // blocks the partial buffer holds
    float *mlp_hist = nullptr;       // per-step loss of the last training run
    int cap_hist_loss = 0;
    long long mlp_t = 0;             // Adam steps taken since the weights were set
    uint32_t *sm_next = nullptr;     // per-SM tile counters of the persistent passes (1024)

    // batched boxes: nbox independent periodic unit boxes in one particle set
    int nbox = 0;                    // 0: one box (no box ids)
    int cap_box = 0;                 // boxes the per-box arrays hold
    int cap_bpart = 0;               // particles the per-particle box arrays hold
    int32_t *box_start = nullptr;    // [nbox+1] caller rows of each box (= sorted slots, box-major)
    int32_t *box_in = nullptr;       // box of each caller row
    int32_t *sbox = nullptr;         // box of each sorted slot
    int32_t *sbox_tmp = nullptr;     // box of each slot of the previous build (rebuild input)
    uint32_t *mkey = nullptr;        // Morton keys in input order during a batched sort
    uint32_t *node_box = nullptr;    // tree nodes: lowest box | highest box << 16
    int cap_node_box = 0;
    double *dtb = nullptr;           // time step of each box (the step's dt for one box)
    unsigned long long *box_dtmin = nullptr;   // per-box CFL minimum (float bits)
    double *box_red = nullptr;       // per-box FP64 diagnostics, 8 per box
    int32_t *fcnt = nullptr;         // occupancy of the feature grid (8^7 cells)
    uint32_t *sel = nullptr;         // row selection: flags and their scan (2 x cap_sel)
    int cap_sel = 0;

    // autotuner of the list passes (variant per pass; -1 = the built-in default)
    int tune_on = 0;
    int tune_done[16] = {0};
    int tune_choice[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    float tune_ms[16] = {0};
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    int32_t *tile_order = nullptr;   // tiles by decreasing pair-set list length
    int cap_order = 0;

    // CUDA graphs of the steady-state step (two: the step swaps state buffers)
    int graph_mode = 0;              // set while a step is captured: no host syncs, no growth
    cudaStream_t gstream = nullptr;  // capture stream
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaEvent_t gev[2] = {nullptr, nullptr};
    long long glaunch[2] = {0, 0};   // kernels in each graph
    long long gcaptures = 0, greplays = 0, grecoveries = 0;
    unsigned long long gkey[2] = {0, 0};   // fingerprint of what each graph captured
    float4 *bk_pos = nullptr, *bk_vel = nullptr;   // state before a run of replayed steps
    int cap_bk = 0;
    unsigned long long alloc_gen = 0;   // bumped by every device (re)allocation

    // recursive coordinate bisection (tile_order 2): per-slot and per-segment scratch
    int cap_rcb = 0, cap_rcb_seg = 0;
    int32_t *rcb_a = nullptr, *rcb_id = nullptr, *rcb_size = nullptr;
    uint32_t *rcb_bin = nullptr, *rcb_f = nullptr, *rcb_lo = nullptr, *rcb_hi = nullptr, *rcb_pick = nullptr;
    uint32_t *rcb_hist = nullptr;

    // hierarchical time bins (the tiles are the leaves; per-tile and sorted per-particle arrays)
    int cap_htb = 0;                 // tiles the per-tile arrays hold
    int cap_htbp = 0;                // particles the per-particle arrays hold
    int32_t *tlev = nullptr;         // level of each leaf
    int32_t *tt0 = nullptr;          // tick its current step started
    int32_t *tlen = nullptr;         // ticks of its current step
    int32_t *twake = nullptr;        // level a passive leaf is raised to by its active neighbours
    uint32_t *tflag = nullptr, *tscan = nullptr;   // active flags and their exclusive scan
    int32_t *tact = nullptr;         // the active leaves of the current tick
    float *du_open = nullptr;        // energy rate of each particle's opening kick
    float *hc = nullptr;             // closing half-kick duration at the cycle end (sorted)
    const int32_t *act = nullptr;    // set: walk, tile lists and list passes cover these tiles only
    int nact = 0;

    // launch accounting and per-pass event timing
    long long launches = 0;
    int prof_on = 0;
    int prof_n = 0;
    int prof_cap = 0;
    cudaEvent_t *prof_ev = nullptr;   // 2 per record
    int *prof_id = nullptr;
};

// ----------------------------------------------------------------- host helpers

int crk_set_error(crk_ctx *ctx, int code, const char *fmt, ...);
int crk_check_cuda(crk_ctx *ctx, cudaError_t e, const char *what);
int crk_ensure_particles(crk_ctx *ctx, int n);
int crk_ensure_lists(crk_ctx *ctx, long long ng, long long nu);
int crk_ensure_pair_once(crk_ctx *ctx);
int crk_ensure_entries(crk_ctx *ctx, long long n_ent, long long n_force);
int crk_grow_forces_keep(crk_ctx *ctx, long long n_force);
int crk_sync_counters(crk_ctx *ctx, cudaStream_t s);

#define CRK_CUDA(ctx, call)                                                      \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return crk_check_cuda((ctx), e_, #call);         \
    } while (0)

#define CRK_LAUNCH_CHECK(ctx, what)                                              \
    do {                                                                         \
        cudaError_t e_ = cudaGetLastError();                                     \
        if (e_ != cudaSuccess) return crk_check_cuda((ctx), e_, (what));        \
    } while (0)

// internal entry points shared between translation units (sorted-order data)
namespace crk {
enum { PROF_P1 = 0, PROF_PN = 1, PROF_P2 = 2, PROF_P3 = 3, PROF_P4 = 4, PROF_P5 = 5, PROF_BUILD = 6,
       PROF_LISTS = 7, PROF_MLP_FWD = 8, PROF_MLP_TRAIN = 9, PROF_DENS = 10, PROF_NPASS = 11 };
constexpr int TUNE_P5_DUAL = 15;   // the autotuner's record of the two-kick P5 pass
constexpr int NVAR = CRK_TUNE_NVARIANT;   // list-pass variants (lvariant)
void mlp_free(crk_ctx *ctx);
void htb_free(crk_ctx *ctx);
int unconverged_tiles(crk_ctx *ctx, cudaStream_t s);   // tiles with flags == 0 -> ctx->tact (crk_htb.cu)
void rcb_free(crk_ctx *ctx);
void graph_free(crk_ctx *ctx);
void prof_begin(crk_ctx *ctx, int id, cudaStream_t s);
void prof_end(crk_ctx *ctx, cudaStream_t s);
int build_cells_sorted(crk_ctx *ctx, int n, const float4 *pos_h, const int32_t *order,
                       cudaStream_t s, const int32_t *box_of_input = nullptr);
int ensure_boxes(crk_ctx *ctx, int n, int nbox);
int load_boxes(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, cudaStream_t s);
int rebuild_lists(crk_ctx *ctx, cudaStream_t s);
int build_tree(crk_ctx *ctx, cudaStream_t s);
int finish_build(crk_ctx *ctx, cudaStream_t s);
int cell_level_host(const crk_ctx *ctx);
int run_volumes(crk_ctx *ctx, cudaStream_t s);
int run_lists(crk_ctx *ctx, cudaStream_t s);
int run_export_lists(crk_ctx *ctx, int mode, const long long *off, int32_t *out, cudaStream_t s);
int scan_u32(crk_ctx *ctx, const uint32_t *in, uint32_t *out, int count, cudaStream_t s);
int run_neighbours(crk_ctx *ctx, int mode, int32_t *cnt, uint32_t *hash, cudaStream_t s);
int run_corrections(crk_ctx *ctx, bool with_gradv, cudaStream_t s);
int run_density(crk_ctx *ctx, cudaStream_t s);
int run_forces(crk_ctx *ctx, cudaStream_t s);
int run_compatible(crk_ctx *ctx, cudaStream_t s, const unsigned long long *skip = nullptr);
int run_compatible_dual(crk_ctx *ctx, const double *dtn, const int32_t *sbox, cudaStream_t s);
int evaluate(crk_ctx *ctx, cudaStream_t s);   // P1..P4 and per-particle time steps (crk_step.cu)
int propose_sorted(crk_ctx *ctx, int n, float4 *pos, const GvRec *gv, const float *Nn, float dt, float tol,
                   cudaStream_t s);   // learned h proposal in sorted order (crk_mlp.cu)
int gather_rows(crk_ctx *ctx, const void *in, void *out, int width_words, cudaStream_t s);
int scatter_rows(crk_ctx *ctx, const void *in, void *out, int width_words, cudaStream_t s);
inline int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }
}  // namespace crk

// ----------------------------------------------------------------- device helpers

namespace crk {

__device__ __forceinline__ uint32_t spread3(uint32_t v) {   // 10 bits -> every 3rd bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t morton30(uint32_t qx, uint32_t qy, uint32_t qz) {
    return spread3(qx >> 22) | (spread3(qy >> 22) << 1) | (spread3(qz >> 22) << 2);
}

// Index along the Hilbert curve through the 2^10 cells per axis of the top 10
// fixed-point bits (Skilling's transposed form: the axes are rotated and
// reflected level by level into the curve's transposed index, which is Gray
// decoded and interleaved, x most significant).  Like the Morton key, a
// prefix of 3k bits names a level-k cell, but consecutive cells along the
// curve always share a face, so runs of consecutive particles stay compact.
__device__ __forceinline__ uint32_t hilbert30(uint32_t qx, uint32_t qy, uint32_t qz) {
    uint32_t X[3] = {qx >> 22, qy >> 22, qz >> 22};
#pragma unroll
    for (uint32_t Q = 1u << 9; Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
#pragma unroll
    for (uint32_t Q = 1u << 9; Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
    return spread3(X[2] ^ t) | (spread3(X[1] ^ t) << 1) | (spread3(X[0] ^ t) << 2);
}

// floor(s * 2^32) for s in [0,1): the product is exact, truncation is floor.
__device__ __forceinline__ uint32_t to_fixed(float s) {
    return (uint32_t)__float2ull_rz(s * 4294967296.0f);
}

// squared fixed-point distance of a minimum-image separation (exact)
__device__ __forceinline__ unsigned long long r2_fixed(int dx, int dy, int dz) {
    return (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
           (unsigned long long)((long long)dz * dz);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace crk
