/*
 * crk.h -- C ABI of the GB300 CRKSPH pair-interaction engine.
 *
 * The engine runs the particle-pair passes of the conservative reproducing-
 * kernel SPH (CRKSPH) scheme used by CRK-HACC (arXiv 2202.02840): volumes,
 * reproducing-kernel corrections, velocity gradients, corrected-kernel
 * momentum and energy pair sums with limited artificial viscosity, and the
 * compatible-energy update, on one GPU (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Units: natural units (a = 1, adot = 0, p = v), periodic unit cube.
 *  - Particle arrays are caller-owned DEVICE pointers, length n, in the
 *    caller's particle order (array-of-records, row-major):
 *      pos_h  float[4n]  (x, y, z, h); x,y,z in [0,1), 0 < h < 1/3
 *      vel_u  float[4n]  (vx, vy, vz, u)
 *      mass   float[n]
 *      V, Nngb, A, dudt, vsig, qmax, du      float[n]
 *      B, gradA, accel, vel_before, vel_after float[3n]
 *      gradB  float[9n]  [i][alpha][gamma] = d B^alpha / d x^gamma
 *      gradv  float[9n]  [i][alpha][beta]  = d v^alpha / d x^beta
 *    All device pointers must be 16-byte aligned and must not alias each
 *    other unless stated.
 *  - Library-owned memory (sorted particle copies, sort scratch, tiles, the
 *    tile tree and interaction lists) belongs to the crk_ctx; it is allocated
 *    by crk_create / grown by crk_build_cells and freed by crk_destroy.
 *  - Streams: every call enqueues its work on `stream` (a cudaStream_t, NULL =
 *    legacy default stream) and returns without waiting, except where a call
 *    says it synchronises.  Outputs are valid once the stream reaches them.
 *  - Errors: functions return CRK_OK (0) or a negative CRK_E* code; the
 *    message of the last failure is available from crk_last_error(ctx).  A
 *    call that fails leaves its outputs unspecified.  Device-side failures
 *    (invalid inputs found by a kernel, exhausted capacity) are reported by
 *    the next synchronising call.
 *
 * Paper readings used at this boundary (where the paper is silent):
 *  - neighbour predicate: positions and h in uint32 fixed point q =
 *    floor(s 2^32), H = floor(h 2^32); minimum-image integer separation;
 *    gather(i) = {j : |dq|^2 < H_i^2} (self included); pair set =
 *    {(i,j), i != j : |dq|^2 < max(H_i, H_j)^2}; x_ij = dq 2^-32.
 *  - gradients in eq:gRK are taken with respect to the evaluation point at
 *    fixed h and fixed neighbour volumes; grad W^R_ji uses particle j's
 *    coefficients with x_ji = -x_ij.
 *  - rho_i = m_i / V_i; P = (gamma - 1) rho u; c_s = sqrt(gamma P / rho).
 */
#ifndef CRK_H
#define CRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRK_OK 0
#define CRK_EINVAL (-1)     /* invalid argument or invalid particle data */
#define CRK_ENOMEM (-2)     /* device allocation failed */
#define CRK_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define CRK_ETIMEOUT (-4)   /* reserved: no entry point returns it (no kernel waits on another) */
#define CRK_ENONCONV (-5)   /* the h fixed-point iteration did not converge */
#define CRK_ECAPACITY (-6)  /* a fixed-capacity buffer overflowed */
#define CRK_ESTATE (-7)     /* call out of order (e.g. a pass before crk_build_cells) */

typedef struct crk_ctx crk_ctx;

/* Method and engine parameters; crk_default_params fills the paper's values. */
typedef struct {
    double gamma;     /* adiabatic index, 5/3 (Sec. 1.1, eq:EOS) */
    double n_h;       /* particles per smoothing length, 4 (Sec. 2.6) */
    double N_res;     /* target neighbour count, 268 (Sec. 2.6, eq:hi) */
    double C_l, C_q;  /* viscosity coefficients 2, 1 (eq:visc) */
    double eps;       /* 0.1 (eq:mu) */
    double eta_crit;  /* 1/n_h (eq:phiad) */
    double eta_fold;  /* 0.2/n_h (eq:phiad) */
    double C_cfl;     /* 0.25 (Sec. 2.1 time-step criteria) */
    double zeta;      /* 4 (Sec. 2.1, c_sq = sqrt(zeta Q / rho)) */
    double h_min;     /* lower clamp of the evolved h (box units) */
    double h_max;     /* upper clamp of the evolved h (< 1/3) */
    double dt_max;    /* cap of the CFL time step */
    double a;         /* cosmic scale factor (Sec. 1.1); 1 = a static box.  The state's
                         velocity column then holds p = a^2 dx/dt = a v (v peculiar) */
    double adot;      /* da/dt; 0 = a static box.  a and adot enter eq:mom (a^2), eq:eng
                         (1/(2a^2), dx/dt = p/a^2), eq:compEng2 (1/(2a^4)), eq:mu (h^/a,
                         u^ = v^ + adot x), the signal velocity ((adot/a) x), eq:gradv (of
                         v = p/a), the drift (p/a^2), the expansion term of eq:CosmoEngEqn
                         and the time-step criteria; crk_set_expansion changes them */
    int precision;    /* 0 = plain FP32 (FP32 sums, FP32 3x3 inverse);
                         1 = mixed (default): FP32 pair sums, compensated momentum
                             and energy accumulation, moments formed and the 3x3
                             system solved in FP64;
                         2 = mixed with compensated moment and grad-v sums too;
                         3 = mode 2 with every pair term of the moments carried in
                             float-float (exact separation and integer r^2, an exact
                             t = 1 - eta, error-free products): B, grad A, grad B
                             to ~1e-8 of their RMS even where the moment sums cancel
                             (lattice-like neighbourhoods), at about twice P2's cost */
    int kmax;         /* finest chaining-mesh level reported by crk_cells (<= 7) */
    int tile_order;   /* order of the particles that cuts them into 32-particle tiles:
                         0 = Morton (default; the chaining-mesh order of Sec. 2.3,
                             the only one crk_cells reports),
                         1 = Hilbert curve (same cells, no jumps between them),
                         2 = recursive coordinate bisection (the paper's leaves) */
    int density;      /* 0 = rho = m/V (default); 1 = the RK-corrected sum
                         rho_i = sum_{j in gather(i)} m_j W^R_ij (eq:RK), self included */
    int h_mode;       /* smoothing length in crk_step / crk_steps (one box):
                         0 = evolved (default, Sec. 2.6): one eq:thacker update of each
                             evaluation's count carries h to the next step;
                         1 = eq:hi solved before every evaluation by the fixed-point
                             iteration of crk_h_iterate (tolerance h_tol, at most h_max_it
                             P1 passes), started from the state's h;
                         2 = as 1, started from the learned proposal (crk_h_propose; the
                             network weights must be set): the first P1 judges and the
                             proposal replaces the first update.
                         In modes 1 and 2 the state keeps the solved h (no eq:thacker
                         update after the evaluation), steps run eagerly (never from a
                         CUDA graph: the solve reads its convergence on the host), and
                         crk_step_batched returns CRK_ESTATE. */
    int h_max_it;     /* iteration cap of h_mode 1 and 2 (default 50) */
    float h_tol;      /* |Delta_N - 1| tolerance of h_mode 1 and 2 (default 1e-4) */
    int rcb_leaf;     /* tile_order 2: particles per bisection leaf, 32 (default: one
                         tile), 128 or 256 (the paper's N_ppl range, Sec. 2.3: a leaf's tiles are
                         cut from the order the splits leave inside it) */
    int pair_form;    /* how P4 and P5 visit the pair set when every tile is evaluated:
                         0 = directed (default): every ordered pair (i, j) is evaluated
                             from its i side (twice per unordered pair; F_ji = -F_ij
                             bitwise);
                         1 = pair-once: each unordered pair is evaluated once,
                             by the particle with the lower sorted index, and j's share
                             (-F_ij, its eq:eng and eq:compEng terms, its Q, the signal
                             velocity) is summed per tile pair and added to j's sums in a
                             fixed order.  Same terms bitwise, another summation order:
                             the results differ from form 0 by rounding only, and repeat
                             bitwise from run to run.  Slower than form 0 on GB300
                             (its lanes wait on one another); kept as the measured
                             alternative.  Passes over a subset of tiles (time bins)
                             always use form 0. */
} crk_params;

/* Per-step diagnostics (host memory), all reductions in FP64. */
typedef struct {
    double dt;            /* time step used */
    double dt_next;       /* CFL time step of the evaluation at the end of the step */
    double E_kin, E_int;  /* sum 1/2 m v^2, sum m u after the step */
    double P[3];          /* total momentum sum m v after the step */
    long long pairs_gather;  /* |gather(i)| - 1 summed over i, last evaluation */
    long long pairs_union;   /* ordered pairs of the pair set, last evaluation */
    long long h_iterations;  /* h_mode 1, 2: P1 passes of the step's eq:hi solve (else 0) */
    long long h_unconverged; /* h_mode 1, 2: particles still outside h_tol after them */
} crk_diag;

/* Fill *p with the paper's values (see crk_params).  Never fails for p != NULL. */
int crk_default_params(crk_params *p);

/* Create an engine on the current CUDA device.  *out receives the context.
 * CRK_EINVAL for NULL pointers or parameters out of range, CRK_ECUDA/ENOMEM
 * if the device cannot be used. */
int crk_create(const crk_params *p, crk_ctx **out);

/* Free every library-owned buffer.  Synchronises the device. */
int crk_destroy(crk_ctx *ctx);

/* Message of the last failed call on ctx (static storage inside ctx). */
const char *crk_last_error(const crk_ctx *ctx);

/* Wait for `stream`, then report device-side errors recorded since the last
 * synchronising call (CRK_EINVAL for invalid particles, CRK_ECAPACITY ...). */
int crk_sync(crk_ctx *ctx, void *stream);

/* Chaining-mesh binning and interaction lists (Sec. 2.3 short-range solver
 * data structures; D1-D4 analogue): fixed-point keys, 30-bit Morton keys,
 * stable LSD radix sort, sorted particle copies, tiles of 32 consecutive
 * particles with fixed-point bounding boxes and max H, an implicit binary
 * tree over tiles, and per-tile interaction lists for the gather predicate and
 * for the pair set.  pos_h is read, never written.  Synchronises `stream`
 * once to size the lists (grows them as needed).  CRK_EINVAL if any
 * coordinate is outside [0,1) or non-finite, or h is not in (0, 1/3). */
int crk_build_cells(crk_ctx *ctx, int n, const float *pos_h, void *stream);

/* Binning of the last build, for inspection (device outputs, may be NULL):
 *  keys[n]      30-bit Morton keys in sorted order (x in bit 0 of each triple,
 *               from the top 10 bits of the fixed-point coordinates)
 *  perm[n]      caller index of each sorted slot (stable in the caller index)
 *  cell_start   int[8^k + 1]: first sorted slot whose cell >= c, k = the
 *               chaining-mesh level, the largest k <= kmax with 2^-k >= max h
 * *k_out (host) receives k.  Synchronises `stream`. */
int crk_cells(crk_ctx *ctx, uint32_t *keys, int32_t *perm, int32_t *cell_start, int *k_out,
              void *stream);

/* Counts of the last build (host outputs, may be NULL): number of tiles,
 * per-particle neighbour-list entries of the last list build (0 before the
 * first pass that needs them; includes per-tile padding), and tile pairs of
 * the pair-set tile list.  Synchronises `stream`. */
int crk_build_stats(crk_ctx *ctx, int *ntiles, long long *list_entries,
                    long long *union_tile_pairs, void *stream);

/* Work of the last neighbour-list walk (Sec. 2.3 interaction lists turned into
 * per-particle lists): *lane_tests = evaluations of the exact fixed-point
 * predicate |dq|^2 < H^2 (each lane of a tile tests every particle kept from
 * each candidate tile; invalid lanes of a ragged last tile included), the
 * walk's unit of work.  0 when the last walk wrote no lists.  Synchronises
 * `stream`. */
int crk_walk_stats(crk_ctx *ctx, long long *lane_tests, void *stream);

/* Neighbour sets of the last build, for inspection: mode 0 = gather(i)
 * (self included), mode 1 = the pair set of i.  Device outputs in caller
 * order: count[n] = set size, hash[n] = sum over the set of fmix32(j + 1)
 * modulo 2^32, with j the caller index and fmix32 the MurmurHash3 32-bit
 * finaliser (x ^= x>>16; x *= 0x85ebca6b; x ^= x>>13; x *= 0xc2b2ae35;
 * x ^= x>>16).  Equal (count, hash) for every particle means equal sets up
 * to a 2^-32 collision chance per particle. */
int crk_neighbours(crk_ctx *ctx, int mode, int32_t *count, uint32_t *hash, void *stream);

/* The per-particle neighbour lists that the list passes walk (the walk of the
 * last build; built here if the passes have not built them yet), in caller
 * order, for inspection.  offsets (device, n + 1 long longs) is the exclusive
 * prefix sum of the set sizes of crk_neighbours in the same mode; lists
 * (device, offsets[n] ints) receives particle i's set in
 * lists[offsets[i] .. offsets[i+1]), in the order the passes visit it:
 *   mode 0: gather(i) (eq:vol; self first), each entry the caller index of j
 *           with bit 31 set when i is in gather(j) too (the "j's kernel
 *           reaches i" flag P4 uses);
 *   mode 1: the pair set of i (the gather neighbours, then the others),
 *           caller indices.
 * CRK_ESTATE in a context without lists (the allocation-free volumes). */
int crk_neighbour_lists(crk_ctx *ctx, int mode, const long long *offsets, int32_t *lists, void *stream);

/* P1, eq:vol and eq:hi: n_i = sum_{j in gather(i)} W(|x_ij|, h_i) with the
 * C4 Wendland kernel of eq:C4, V_i = 1/n_i, Nngb_i = 4/3 pi h_i^3 n_i.
 * Outputs V[n], Nngb[n] (Nngb may be NULL).  *pairs (host, may be NULL)
 * receives sum_i (|gather(i)| - 1) and makes the call synchronise. */
int crk_volumes(crk_ctx *ctx, float *V, float *Nngb, long long *pairs, void *stream);

/* P2 + P3.  Moments of W over gather(i) and the reproducing-kernel
 * coefficients of eq:RK / eq:gRK from the moment conditions
 * sum_j V_j W^R_ij = 1, sum_j V_j x_ij W^R_ij = 0 (Sec. 1.2):
 *   B = -m2^-1 m1, A = 1/(m0 + m1.B), grad B = -m2^-1 (grad m1 + grad m2 B),
 *   grad A = -A^2 (grad m0 + B.grad m1 + m1.grad B)
 * (3x3 inverse in FP64 when precision >= 1), then the velocity gradient of
 * eq:gradv, grad v_i = -sum_j V_j (v_i - v_j) (x) grad W^R_ij.
 * Inputs V[n], vel_u[4n]; outputs A, B, gradA, gradB, gradv (gradv may be
 * NULL to skip P3). */
int crk_corrections(crk_ctx *ctx, const float *V, const float *vel_u, float *A, float *B,
                    float *gradA, float *gradB, float *gradv, void *stream);

/* P4, eq:mom and eq:eng with P -> P + Q (eq:visc, eq:mu), the midpoint
 * projection of eq:hatvi and the limiter of eq:phi .. eq:phiad, over the pair
 * set:  accel_i = (1/m_i) sum_j 1/2 V_i V_j (P~_i + P~_j)(grad W^R_ji - grad W^R_ij),
 * dudt_i = (1/m_i) sum_j 1/2 V_i V_j P~_j (v_j - v_i).(grad W^R_ji - grad W^R_ij),
 * vsig_i = max_j max(0, -(v_i - v_j).x_ij/|x_ij|), qmax_i = max_j Q_i of the pair.
 * Inputs as produced by crk_volumes / crk_corrections (caller order).
 * Outputs accel[3n], dudt[n], vsig[n], qmax[n] (vsig, qmax may be NULL).
 * *pairs (host, may be NULL) receives the ordered pair count and makes the
 * call synchronise. */
int crk_forces(crk_ctx *ctx, const float *mass, const float *vel_u, const float *V,
               const float *A, const float *B, const float *gradA, const float *gradB,
               const float *gradv, float *accel, float *dudt, float *vsig, float *qmax,
               long long *pairs, void *stream);

/* P5, compatible energy of eq:compEng .. eq:fij (adot = 0): with F_ij the
 * pair force of crk_forces evaluated on (mass, vel_u, V, A, B, gradA, gradB,
 * gradv) and a kick that took velocities vel_before -> vel_after,
 *   du_i = sum_j f_ij/2 (v_j + v'_j - v_i - v'_i).F_ij/m_i,
 * f_ij from the specific entropies s = P/rho^gamma and the sign of
 * Delta E_ij = 1/2 (v_j + v'_j - v_i - v'_i).F_ij (f = 1/2 if s_i + s_j = 0).
 * Multiply du by the kick's duration to get the energy increment. */
int crk_compatible(crk_ctx *ctx, const float *mass, const float *vel_u, const float *V,
                   const float *A, const float *B, const float *gradA, const float *gradB,
                   const float *gradv, const float *vel_before, const float *vel_after,
                   float *du, void *stream);

/* One hydro step, the velocity-Verlet KDK operator of eq:verletOP (Sec. 2.1)
 * with predicted p_p, u_p and compatible energy (eq:compEng), on the caller's
 * state pos_h[4n], vel_u[4n] (updated in place) and mass[n]:
 *   half kick with the rates of the last evaluation, drift, rebuild,
 *   evaluation P1..P4 at (x1, p_p, u_p), second half kick; h is advanced
 *   by one eq:thacker update of the new evaluation (clamped to
 *   [h_min, h_max]).  The first call (or the first after crk_reset_rates)
 *   evaluates the rates at the initial state.  dt > 0 fixes the step;
 *   dt <= 0 uses the CFL step of the last evaluation (Sec. 2.1 criteria,
 *   capped by dt_max).  diag (host, may be NULL) receives FP64 diagnostics
 *   and makes the call synchronise.  The caller must not reorder or edit the
 *   state between steps without calling crk_reset_rates. */
int crk_step(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double dt,
             crk_diag *diag, void *stream);

/* nsteps KDK steps (as nsteps calls of crk_step with the same dt).  With
 * use_graph = 1 every step after the first of a fresh state is one launch of
 * a CUDA graph of the whole multi-pass step (two graphs: consecutive steps
 * rotate the engine's state buffers), captured once and replayed with no host
 * work between steps.  Nothing can grow inside a replayed step, so before the
 * replays the call gives the neighbour-list columns and the tile-pair lists
 * 50% headroom over the last step's needs (one more eager step applies a new
 * column width) and the stored forces their worst case; each replayed step
 * records whether a capacity was exceeded anyway.  If one was, the call
 * restores the positions and velocities its replays started from and redoes
 * those steps eagerly, the first of them evaluating the rates afresh at the
 * restored state (so, unlike uninterrupted steps, without the predicted
 * rates of R12).  Otherwise the results are bitwise those of eager steps.  A
 * step that cannot be captured runs eagerly.  While crk_autotune is tuning,
 * steps run eagerly until every pass has been tuned.  diag (host, may be
 * NULL) receives the last step's diagnostics.  Synchronises. */
int crk_steps(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, int nsteps, double dt,
              int use_graph, crk_diag *diag, void *stream);

/* crk_steps for batched boxes (box table as for crk_step_batched; dt > 0
 * applies to every box, dt <= 0 gives each box its CFL step). */
int crk_steps_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, float *pos_h, float *vel_u,
                      const float *mass, int nsteps, double dt, int use_graph, void *stream);

/* Graphs captured, graph launches, and replay runs redone eagerly after a
 * capacity overflow, by crk_steps since crk_create (each may be NULL). */
int crk_graph_stats(crk_ctx *ctx, long long *captures, long long *replays, long long *recoveries);

/* Set the scale factor a > 0 and its rate adot for the following calls (see
 * crk_params.a): a step uses them as constants over its duration (the caller
 * passes the values of the step's midpoint).  The cached rates of the last
 * evaluation were computed with the previous values. */
int crk_set_expansion(crk_ctx *ctx, double a, double adot);

/* Forget the cached rates so that the next crk_step evaluates afresh. */
int crk_reset_rates(crk_ctx *ctx);

/* Fixed-point solve of eq:hi by eq:thacker updates (Sec. 2.6): repeat P1 and
 * the Thacker update (clamped to [h_min, h_max]) for every particle not yet
 * converged, until |Delta_N - 1| <= tol for all particles or max_it
 * iterations.  A particle held at a bound that its update points beyond (a
 * particle in a void that would need h > h_max) counts as converged: that is
 * the bound-constrained solution.  Converged particles keep their h.  Reads and
 * updates the h column of pos_h[4n] in place (tiles are rebuilt as h
 * changes).  *iterations (host) receives the iterations used.  Returns
 * CRK_ENONCONV if some particle did not converge.  Synchronises. */
int crk_h_iterate(crk_ctx *ctx, int n, float *pos_h, float tol, int max_it, int *iterations,
                  void *stream);

/* ------------------------------------------------------------------------
 * Hierarchical power-of-two time bins (Sec. 2.1: the hydro subcycles of
 * eq:Usubsub, the criteria Delta y_hyd and Delta y_acc, leaf-level bins, the
 * f_l limiter, parabolic streaming of passive leaves).
 *
 * A cycle advances the state by one base step Delta, cut into 2^L ticks.  The
 * leaves are the 32-particle tiles of the Morton order at the cycle start;
 * they keep their particles for the whole cycle.  A leaf at level l steps
 * 2^(L-l) ticks.  Levels:
 *   particle: the smallest l >= 0 with Delta / 2^l < dt_i (the per-particle
 *     CFL and acceleration criteria of crk_step, compared in FP64); a particle
 *     needing l > L is held at L and counted as unresolved;
 *   leaf: the deepest of its particles, raised by the limiter so that leaves
 *     on each other's interaction list (tile boxes closer than the larger
 *     Hmax) differ by at most f_l levels: at the cycle start to the least
 *     fixed point over all leaves; mid-cycle over the leaves ending a step
 *     (the others held), which also wake every passive neighbour up to at
 *     least their level - f_l (its step then ends at the first tick that is a
 *     multiple of its new step, and its half kick shrinks to match);
 *   a leaf moves to a shallower level one level at a time, at a tick aligned
 *     with the doubled step.
 * Every tick at which some leaf ends its step: all particles stream along
 * x0 + p0 t + a t^2/2 (constant acceleration of their last evaluation), the
 * leaves ending a step evaluate P1..P4 (passive neighbours enter with their
 * streamed x, v, u and last evaluated V, A, B, grad A, grad B, grad v), close
 * their KDK step with compatible energy (eq:verletOP, eq:compEng), advance h
 * by one eq:thacker update and open their next step.  At the last tick every
 * leaf ends its step together; the particles are sorted again and evaluated
 * in full, which is also the evaluation the next cycle (or crk_step) opens
 * with.
 * ---------------------------------------------------------------------- */

typedef struct {
    int ticks;                  /* ticks at which some leaf ended a step (incl. the last) */
    long long evaluations;      /* particle derivative evaluations, incl. the full one at the end */
    long long wakeups;          /* passive leaves raised by the limiter */
    long long unresolved;       /* particle level requests deeper than L (held at L) */
    int leaves;                 /* leaves (tiles) of the cycle */
    int level_count[32];        /* leaves per level at the cycle start */
} crk_htb_stats;

/* One cycle of hierarchical time bins on the caller's state pos_h[4n],
 * vel_u[4n] (updated in place, synchronized at the end) and mass[n].
 * Delta > 0 is the base step, 0 <= L <= 20 the number of levels below it,
 * f_l >= 0 the limiter.  Like crk_step it opens with the cached evaluation
 * of the last step or cycle (evaluating afresh after crk_reset_rates or on a
 * new state) and leaves the evaluation at its end cached.  stats (host, may
 * be NULL).  One box only (CRK_ESTATE after a batched build).  Synchronises
 * once or twice per tick. */
int crk_cycle(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double Delta, int L,
              int f_l, crk_htb_stats *stats, void *stream);

/* The level assignment of a cycle start, on its own: bins pos_h[4n] (as
 * crk_build_cells), takes the per-particle time steps dt[n] (device, caller
 * order) and writes level[n] (device, caller order): the level of each
 * particle's leaf after the limiter's fixed point.  *unresolved (host, may be
 * NULL) receives the count of particle requests deeper than L.  Synchronises. */
int crk_htb_levels(crk_ctx *ctx, int n, const float *pos_h, const float *dt, double Delta, int L, int f_l,
                   int32_t *level, long long *unresolved, void *stream);

/* ------------------------------------------------------------------------
 * Batched boxes.  nbox independent periodic unit boxes in one particle set:
 * box b owns the caller rows [box_start[b], box_start[b+1]) (host array of
 * nbox + 1 ascending ints, box_start[0] = 0, box_start[nbox] = n, nbox <=
 * 65535).  Every box is its own simulation of Sec. 2 in its own unit cube
 * (positions in [0,1), minimum images within the box, its own time step);
 * particles of different boxes never interact.  One launch of each pass
 * covers all boxes, so many small or unevenly occupied boxes cost one set of
 * launches (the persistent P4 pass balances their tiles across the SMs).
 * ---------------------------------------------------------------------- */

/* Bin all boxes (as crk_build_cells, per box).  After it, crk_volumes,
 * crk_corrections, crk_forces, crk_compatible and crk_neighbours work on the
 * batched build with their usual arguments (caller order over all rows);
 * crk_cells returns CRK_ESTATE (its chaining-mesh table describes one box).
 * CRK_EINVAL for a bad box table or invalid particle records.  Synchronises. */
int crk_build_cells_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, const float *pos_h,
                            void *stream);

/* One KDK step of every box (as crk_step, per box): dt (host, nbox doubles,
 * may be NULL) fixes each box's step, <= 0 or NULL selects that box's CFL
 * step.  diag (host, nbox entries, may be NULL) receives each box's FP64
 * diagnostics (pairs_gather and pairs_union are totals over all boxes) and
 * makes the call synchronise.  The box table is reloaded (and the rates
 * re-evaluated) whenever it differs from the previous call's. */
int crk_step_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, float *pos_h, float *vel_u,
                     const float *mass, const double *dt, crk_diag *diag, void *stream);

/* The sorted order of the last build: perm[s] (device, n ints) = the caller
 * row in slot s; tile t holds slots 32t .. 32t + 31.  For every tile_order
 * (crk_cells reports the Morton order with its cell table). */
int crk_order(crk_ctx *ctx, int32_t *perm, void *stream);

/* Per-pass GPU timing, for roofline measurement.  enable = 1 clears the
 * records and starts recording a CUDA event pair around every pass kernel (and
 * around each cell build), on the stream that kernel is launched on; enable = 0
 * stops recording.  At most 4096 records are kept. */
int crk_profile(crk_ctx *ctx, int enable);

#define CRK_PROF_NPASS 11
/* Wait for the recorded events and sum them per pass: ms[k] (milliseconds)
 * and counts[k] (records) for k = 0 P1 volumes, 1 neighbour sets, 2 P2
 * corrections, 3 P3 grad v, 4 P4 forces, 5 P5 compatible energy, 6 cell build
 * (all its kernels), 7 neighbour-list fill, 8 learned-h inference
 * (crk_mlp_forward, or crk_h_propose with its cell count), 9 one training step
 * (gradient and Adam), 10 the RK-corrected density pass; arrays of CRK_PROF_NPASS entries
 * (may be NULL).  P1 is the list-counting walk, which also computes volumes.
 * *total_launches (may be NULL) = kernels launched by ctx since crk_create. */
int crk_profile_read(crk_ctx *ctx, double *ms, long long *counts, long long *total_launches);

/* Autotuner of the list passes (P1, P2, P3, P4, P5).  Each pass has variants
 * that differ only in how its work is laid out on the GPU: how many list
 * entries a lane takes per iteration (1-4, for the passes with small
 * neighbour records), the order tiles are taken in (Morton order over the
 * grid; contiguous tile ranges per SM in a persistent launch; longest
 * pair-set list first) and how many 32-particle tiles share a CTA (1, 2, 4
 * or 8: 32-256 particles).  Every variant visits each particle's list in the
 * same order, so all produce bitwise identical results.  enable = 1 makes the
 * next call of each pass time every variant once (on the stream, with CUDA
 * events; the call synchronises while tuning) and keep the fastest for the
 * context; enable = 0 keeps the choices made and stops tuning. */
int crk_autotune(crk_ctx *ctx, int enable);

/* The variant chosen for each pass k (CRK_PROF_NPASS entries, numbering as in
 * crk_profile_read; -1 = not tuned, the built-in default runs) and its time in
 * ms.  Variants 0-3: Morton order, 1-4 entries per iteration; 4-7: longest
 * list first, 1-4 entries; 8: per-SM tile ranges, 1 entry; 9-12: Morton order
 * with the pass's own entries per iteration and CTAs of 1, 2, 4, 8 tiles;
 * 13-16: 1-4 entries per iteration with the neighbour records of the next
 * iteration read ahead, CTAs of one tile; 17-20: the same with the pass's own
 * CTA width (13-20 for every list pass but P4); 21 (P4 only): the neighbour
 * records brought into shared memory by TMA gathers (tile::gather4 from L2,
 * two stages per warp, an mbarrier per stage), measured 6x slower than the L1
 * forms on GB300 and therefore run only when pinned by crk_tune_set, never
 * by the tuner's sweep; 22 (every list pass but P4): per-SM tile ranges with
 * the pass's own entries per iteration and the records of the next iteration
 * read ahead.  Either array may be NULL. */
int crk_tuning(crk_ctx *ctx, int *variant, float *ms);

/* Number of pass variants (the numbering of crk_tuning). */
#define CRK_TUNE_NVARIANT 23

/* Pin list pass k (numbering as in crk_profile_read: 0 P1, 2 P2, 3 P3, 4 P4,
 * 5 P5, 10 RK density) to variant v (numbering as in crk_tuning; -1: the
 * built-in default) and stop tuning it; for P5, both the one-kick and the
 * two-kick pass.  Every variant gives bitwise the same results, so this only
 * fixes the speed.  A later crk_autotune(ctx, 1) unpins every pass.
 * CRK_EINVAL for another k or v outside [-1, CRK_TUNE_NVARIANT); a variant the
 * pass does not have (P4 has only 0, 4, 8-12) makes the pass's next call
 * return CRK_EINVAL. */
int crk_tune_set(crk_ctx *ctx, int pass, int variant);

/* Largest n accepted by crk_volumes_noalloc. */
#define CRK_NOALLOC_MAX_N 16384

/* P1 volumes (as crk_build_cells followed by crk_volumes) for callers that
 * cannot allocate device memory: applications that own the whole GPU through
 * their own allocator, or that must never call cudaMalloc/cudaFree because
 * those calls can synchronise the device mid-computation.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *
 * pos_h[4n] (device, caller order) in; V[n] and Nngb[n] (device; Nngb may be
 * NULL) out, in caller order.  No context, no allocation: every piece of
 * scratch memory lives in one file-scope __device__ array of about 3.0 MB
 * that every GPU loading this library holds until the process exits.
 *  - n must be in [0, CRK_NOALLOC_MAX_N]; larger n returns CRK_EINVAL.
 *  - CRK_EINVAL also for invalid particle records (as crk_build_cells).
 *  - The first call on a device resolves the array's device address for that
 *    device (cudaGetSymbolAddress) and keeps it for later calls.
 *  - All calls share the array and it keeps the last call's contents; each
 *    call clears what must start at zero.  Calls that overlap on the GPU
 *    (other streams, other host threads) race on it: serialise them.
 *  - The call synchronises `stream` once (to check the binning) and then
 *    enqueues P1 and the output scatter on it.
 *  - CRK_ESTATE if some internal buffer would have had to grow (which would
 *    mean a library allocation); with the fixed sizes above this does not
 *    happen for any n it accepts. */
int crk_volumes_noalloc(int n, const float *pos_h, float *V, float *Nngb, void *stream);

/* ------------------------------------------------------------------------
 * Learned smoothing-length proposal.
 *
 * The paper evolves h by one Thacker update per step (Sec. 2.6, eq:thacker;
 * eq:hi defines the target neighbour count N_res).  Solving eq:hi exactly is
 * the fixed-point iteration of crk_h_iterate; these calls propose its
 * starting point with a small network trained on converged solutions.  The
 * iteration stays in charge: it judges every proposal and corrects it to the
 * same tolerance as without one.
 *
 * Features, 8 per particle, row-major float[8n] in caller order.  Cells are
 * those of the grid of side 2^-kf, kf the largest k in [1, 7] with
 * 64 * 8^k <= n (so that 2^-kf >= 4 N^(-1/3), about one kernel support at
 * N_res); a particle's cell is the top kf bits of its fixed-point
 * coordinates, neighbours wrap periodically (with 2 cells per axis an offset
 * of -1 and +1 reach the same cell and both count):
 *   0 log(1 + own cell count)        1 log(1 + sum of the 6 face cells)
 *   2 log(1 + sum of the 12 edge cells) 3 log(1 + sum of the 8 corner cells)
 *   4 log(1 + sum of all 27 cells)   5 log(h / Delta), Delta = N^(-1/3)
 *   6 dt div v (div v = trace of gradv, dt the step that led to the state;
 *     0 without gradv): the compression h div v made dimensionless by the
 *     step, so that it transfers between resolutions
 *   7 log(Nngb / N_res) (0 without Nngb)
 * Network: y = s_y (W3 . silu(W2 silu(W1 x + b1) + b2) + b3), sizes 8 -> 64
 * -> 64 -> 1, silu(z) = z / (1 + e^-z), s_y = CRK_MLP_YSCALE a fixed output
 * scale (the corrections are of order 1% in log h; the scale keeps the
 * network's own outputs of order one).  Parameters are one FP32 array of
 * CRK_MLP_NPARAM values packed as W1 (64x8, row-major [out][in]), b1 (64),
 * W2 (64x64, [out][in]), b2 (64), W3 (64), b3 (1).  Arithmetic: weights, the
 * features and both hidden activations are rounded to BF16, products are
 * accumulated in FP32 on the tensor cores, biases stay FP32, and silu uses
 * the hardware tanh approximation of the logistic function.
 * Target of training: log(h_conv / h_ref) (h_ref below); loss: mean squared error over the
 * batch; optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32
 * master weights, which the context owns.
 * ---------------------------------------------------------------------- */
#define CRK_MLP_NPARAM 4801
#define CRK_MLP_NFEAT 8
#define CRK_MLP_YSCALE 0.015625f

/* Copy the network parameters in (w: CRK_MLP_NPARAM floats, host or device)
 * and reset the Adam state.  Must precede every other crk_mlp / crk_h_propose
 * call (CRK_ESTATE otherwise). */
int crk_mlp_set_weights(crk_ctx *ctx, const float *w, void *stream);

/* Copy the current FP32 master weights out (host or device pointer). */
int crk_mlp_get_weights(crk_ctx *ctx, float *w, void *stream);

/* Features of n particles.  pos_h[4n] in; gradv[9n] and Nngb[n] (device, may
 * be NULL) and the step dt >= 0 in; feat[8n] out.  With pos_conv[4n] (the same particles with the
 * converged h in the w column) also target[n] = log(h_conv / h_ref), where
 * h_ref = h_prev (N_res / Nngb)^(1/3) with Nngb (the constant-density
 * solution of eq:hi, which the proposal starts from) and h_ref = h_prev
 * without; pos_conv and target are both NULL or both set.  CRK_EINVAL for
 * coordinates outside [0,1) or h outside (0,1).  Synchronises `stream` once
 * to check the records. */
int crk_h_features(crk_ctx *ctx, int n, const float *pos_h, const float *gradv, const float *Nngb, float dt,
                   const float *pos_conv, float *feat, float *target, void *stream);

/* Network output y[n] (device) for the feature rows feat[8n] (device). */
int crk_mlp_forward(crk_ctx *ctx, int n, const float *feat, float *y, void *stream);

/* Proposal, in place: the h column of pos_h[4n] (device) becomes
 * clamp(h_ref exp(y), h_min, h_max), y the network output for the particle's
 * features (computed in the same kernel from pos_h, gradv, Nngb, dt as for
 * crk_h_features) and h_ref as there: the network corrects the
 * constant-density estimate h (N_res / Nngb)^(1/3) (h without Nngb).  A
 * particle whose Nngb already satisfies |(N_res / Nngb)^(1/3) - 1| <= tol
 * keeps its h (the judge of crk_h_iterate).  Synchronises `stream` once to
 * check the records; on CRK_EINVAL the h column is unspecified. */
int crk_h_propose(crk_ctx *ctx, int n, float *pos_h, const float *gradv, const float *Nngb, float dt, float tol,
                  void *stream);

/* One full-batch step over the n rows feat[8n], target[n] (device): the
 * gradient of the mean squared error goes to grad[CRK_MLP_NPARAM] (device,
 * may be NULL) and the loss to loss[1] (device, may be NULL); then, for
 * lr > 0, one Adam update of the weights (lr = 0 leaves them unchanged, which
 * makes this the gradient evaluation). */
int crk_mlp_train_step(crk_ctx *ctx, int n, const float *feat, const float *target, float lr, float *grad,
                       float *loss, void *stream);

/* Rows that the proposal acts on: rows[0..*count) (device out, capacity n)
 * receives, in increasing order, base + i for every i with
 * |(N_res / Nngb[i])^(1/3) - 1| > tol (Nngb device, n floats); *count
 * (host) their number.  base offsets the indices into a data set that
 * concatenates several snapshots.  Synchronises `stream`. */
int crk_h_select(crk_ctx *ctx, int n, const float *Nngb, float tol, int base, int32_t *rows, int *count,
                 void *stream);

/* `steps` Adam steps on batches of `batch` rows drawn with replacement by a
 * counter-based generator (SplitMix64 of seed and the global step count, so
 * that successive calls continue the sequence) from the rows feat[8n],
 * target[n] (device): from all n rows when rows is NULL, else from the
 * n_rows row indices rows[] (device, each in [0, n)).  loss_hist (host,
 * `steps` floats, may be NULL) receives the loss of each batch; with
 * loss_hist the call synchronises. */
int crk_mlp_train(crk_ctx *ctx, int n, const float *feat, const float *target, const int32_t *rows, int n_rows,
                  int batch, int steps, float lr, unsigned long long seed, float *loss_hist, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CRK_H */
