// crk_step.cu -- the hydro step of CRK-HACC Sec. 2.1 (velocity-Verlet KDK
// operator eq:verletOP with predicted p_p, u_p and the compatible energy of
// eq:compEng), the time-step criteria of Sec. 2.1 (natural units, no gravity),
// the evolved smoothing length of Sec. 2.6 (eq:thacker) and its fixed-point
// solve, and FP64 conservation diagnostics.
//
// Between steps the engine keeps the last evaluation (sorted particle copies,
// A, B, grad A, grad B, grad v, accelerations, evaluation velocities) so the
// first half kick of the next step reuses it: one force evaluation per step.
#include "crk_internal.cuh"

#include <math.h>
#include <string.h>

#include <vector>

namespace crk {

static float bits_to_float(uint32_t b) {
    float f;
    memcpy(&f, &b, sizeof(f));
    return f;
}

struct StepConsts {
    float gamma, gm1, inv_nh, C_cfl, zeta, N_res, h_min, h_max;
    double dt_max;
    // comoving variables (1, 1, 0, 0 in a static box)
    float inv_a, inv_a2, adot;
    float E;   // (adot/a)(3(gamma-1) + 2): expansion term of eq:CosmoEngEqn
    int keep_h;   // h_mode >= 1: the state keeps the solved h of its evaluation
};

static StepConsts step_consts(const crk_params &p) {
    StepConsts c;
    c.gamma = (float)p.gamma;
    c.gm1 = (float)(p.gamma - 1.0);
    c.inv_nh = (float)(1.0 / p.n_h);
    c.C_cfl = (float)p.C_cfl;
    c.zeta = (float)p.zeta;
    c.N_res = (float)p.N_res;
    c.h_min = (float)p.h_min;
    c.h_max = (float)p.h_max;
    c.dt_max = p.dt_max;
    c.inv_a = (float)(1.0 / p.a);
    c.inv_a2 = (float)(1.0 / (p.a * p.a));
    c.adot = (float)p.adot;
    c.E = (float)(p.adot / p.a * (3.0 * (p.gamma - 1.0) + 2.0));
    c.keep_h = p.h_mode >= 1;
    return c;
}

// Per-particle time step (Sec. 2.1, pure hydro so r_soft -> inf and the total
// acceleration is (1/a^2) dp/dt):
// v_max = max(v_sig, c_s, sqrt(zeta Q/rho), (h_hat/a) |tr grad v + 3 adot|),
// dt_i = min(C_CFL h_hat / v_max, sqrt(h_hat / |a_tot|)); global min as float bits.
__global__ void k_cfl(int n, StepConsts c, const float *__restrict__ hs, const float *__restrict__ V,
                      const float *__restrict__ mass, const float4 *__restrict__ vel,
                      const float4 *__restrict__ acc, const float2 *__restrict__ vq,
                      const GvRec *__restrict__ gv, unsigned long long *dtmin, const int32_t *__restrict__ sbox,
                      float *__restrict__ dt_out, const float *__restrict__ rho_in) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    float dt = 3.0e38f;
    if (s < n) {
        float hh = hs[s] * c.inv_nh;
        float rho = rho_in ? rho_in[s] : mass[s] / V[s];
        float u = vel[s].w;
        float cs = sqrtf(fmaxf(c.gamma * c.gm1 * u, 0.f));
        float2 q = vq[s];
        float csq = sqrtf(fmaxf(c.zeta * q.y / rho, 0.f));
        GvRec g = gv[s];
        float div = fabsf(fmaf(3.f, c.adot, g.g0.x + g.g1.x + g.g2.x)) * c.inv_a;
        float vmax = fmaxf(fmaxf(q.x, cs), fmaxf(csq, hh * div));
        if (vmax > 0.f) dt = fminf(dt, c.C_cfl * hh / vmax);
        float4 a = acc[s];
        float am = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z) * c.inv_a2;
        if (am > 0.f) dt = fminf(dt, sqrtf(hh / am));
        dt_out[s] = dt;   // per particle, for the time bins
    }
    if (sbox) {   // batched boxes: one minimum per box (one atomic per box a warp touches)
        const int b = s < n ? sbox[s] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        unsigned m = __float_as_uint(dt);
        for (int k = 0; k < 32; k++) {
            const unsigned mk = __shfl_sync(0xffffffffu, m, k);
            if (((peers >> k) & 1u) && mk < m) m = mk;
        }
        if (b >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(dtmin + b, (unsigned long long)m);
        return;
    }
    unsigned m = __reduce_min_sync(0xffffffffu, __float_as_uint(dt));
    if ((threadIdx.x & 31) == 0) atomicMin(dtmin, (unsigned long long)m);
}

__global__ void k_fill_ull(int count, unsigned long long v, unsigned long long *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) out[k] = v;
}

// dt of this step for each box: the requested dt, or min(CFL dt, dt_max);
// req (device, one per box) may be null, dt_req then applies to every box
__global__ void k_pick_dt(int nbox, double dt_req, const double *req, double dt_max,
                          const unsigned long long *dtmin, double *dtb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    double dt = req ? req[b] : dt_req;
    if (!(dt > 0.0)) {
        dt = (double)__uint_as_float((uint32_t)dtmin[b]);
        if (!(dt < dt_max)) dt = dt_max;
    }
    dtb[b] = dt;
}

// The opening kick of a step may take the energy rates that the previous
// step's dual P5 pass formed ahead (CNT_NEXT_OK), but only if they were formed
// for exactly this step's dt in every box; the flag is consumed either way.
__global__ void k_next_check(int nbox, const double *__restrict__ dtb, const double *__restrict__ dtn,
                             unsigned long long *cnt) {
    __shared__ int differ;
    if (threadIdx.x == 0) differ = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nbox; b += blockDim.x)
        if (dtb[b] != dtn[b]) differ = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        cnt[CNT_SKIP] = (cnt[CNT_NEXT_OK] && !differ) ? 1ull : 0ull;
        cnt[CNT_NEXT_OK] = 0ull;
    }
}

// the opening kick's energy rates when its P5 pass was skipped
__global__ void k_take_next(int n, const unsigned long long *cnt, const float *__restrict__ du_next,
                            float *__restrict__ du) {
    if (!cnt[CNT_SKIP]) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) du[s] = du_next[s];
}

__global__ void k_set_next_ok(unsigned long long *cnt) { cnt[CNT_NEXT_OK] = 1ull; }

// dt of slot s: its box's (one box: dtb[0])
__device__ __forceinline__ double slot_dt(const double *dtb, const int32_t *sbox, int s) {
    return dtb[sbox ? sbox[s] : 0];
}

// first half kick of eq:verletOP: p_1/2 = p + a dt/2; vb = p, va = p_1/2
__global__ void k_kick1(int n, const double *sc, const int32_t *__restrict__ sbox, const float4 *__restrict__ st_vel, const float4 *__restrict__ acc,
                        float4 *__restrict__ vb, float4 *__restrict__ va) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h = (float)(0.5 * slot_dt(sc, sbox, s));
    float4 v = st_vel[s], a = acc[s];
    vb[s] = make_float4(v.x, v.y, v.z, 0.f);
    va[s] = make_float4(fmaf(h, a.x, v.x), fmaf(h, a.y, v.y), fmaf(h, a.z, v.z), 0.f);
}

// u_1/2 = u + (du - E u) dt/2; predictor p_p = p_1/2 + a dt/2,
// u_p = (u_1/2 + du dt/2) / (1 + E dt/2); drift x1 = x + p_1/2 dt / a^2
// (periodic wrap into [0,1)).  The expansion term -E u of eq:CosmoEngEqn
// enters the opening half kick explicitly and the closing ones implicitly:
// the trapezoidal rule over the step (E = 0 in a static box).
__global__ void k_half_drift(int n, const double *sc, const int32_t *__restrict__ sbox, StepConsts c,
                             float4 *__restrict__ st_pos, float4 *__restrict__ st_vel,
                             float4 *__restrict__ st_half, const float4 *__restrict__ va,
                             const float4 *__restrict__ acc, const float *__restrict__ du) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float dt = (float)slot_dt(sc, sbox, s), h = 0.5f * dt;
    float4 v = st_vel[s], ph = va[s], a = acc[s];
    float uh = fmaf(h, fmaf(-c.E, v.w, du[s]), v.w);
    st_half[s] = make_float4(ph.x, ph.y, ph.z, uh);
    st_vel[s] = make_float4(fmaf(h, a.x, ph.x), fmaf(h, a.y, ph.y), fmaf(h, a.z, ph.z),
                            fmaf(h, du[s], uh) / fmaf(h, c.E, 1.f));
    float4 p = st_pos[s];
    const float dx = dt * c.inv_a2;
    float x[3] = {fmaf(dx, ph.x, p.x), fmaf(dx, ph.y, p.y), fmaf(dx, ph.z, p.z)};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        x[k] -= floorf(x[k]);
        if (x[k] >= 1.f) x[k] = 0.f;
        if (x[k] < 0.f) x[k] = 0.f;
    }
    st_pos[s] = make_float4(x[0], x[1], x[2], p.w);
}

// new slot s takes old slot idx[s]
__global__ void k_permute3(int n, const int32_t *__restrict__ idx, const float4 *__restrict__ a,
                           float4 *__restrict__ ao, const float4 *__restrict__ b, float4 *__restrict__ bo,
                           const float4 *__restrict__ c, float4 *__restrict__ co) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int o = idx[s];
    ao[s] = a[o];
    bo[s] = b[o];
    co[s] = c[o];
}

// second half kick: p1 = p_1/2 + a1 dt/2; vb = p_1/2, va = p1
__global__ void k_kick2(int n, const double *sc, const int32_t *__restrict__ sbox, const float4 *__restrict__ st_half, const float4 *__restrict__ acc,
                        float4 *__restrict__ vb, float4 *__restrict__ va) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h = (float)(0.5 * slot_dt(sc, sbox, s));
    float4 v = st_half[s], a = acc[s];
    vb[s] = make_float4(v.x, v.y, v.z, 0.f);
    va[s] = make_float4(fmaf(h, a.x, v.x), fmaf(h, a.y, v.y), fmaf(h, a.z, v.z), 0.f);
}

// final state: v1 = va, u1 = u_1/2 + du dt/2; h advanced by eq:thacker
__global__ void k_finish(int n, const double *sc, const int32_t *__restrict__ sbox, StepConsts c, const float4 *__restrict__ st_half,
                         const float4 *__restrict__ va, const float *__restrict__ du, const float *__restrict__ Nn,
                         const float *__restrict__ hs, float4 *__restrict__ st_vel, float4 *__restrict__ st_pos) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h = (float)(0.5 * slot_dt(sc, sbox, s));
    float4 a = va[s];
    st_vel[s] = make_float4(a.x, a.y, a.z, fmaf(h, du[s], st_half[s].w) / fmaf(h, c.E, 1.f));
    float hn = hs[s];
    if (!c.keep_h) {   // the evolved h: one eq:thacker update of the evaluation's count
        float d = cbrtf(c.N_res / Nn[s]);
        float lam = d < 1.f ? 0.2f * (1.f + d * d) : 0.2f * (1.f + 1.f / (d * d * d));
        hn = fminf(fmaxf(hs[s] * (1.f - lam + lam * d), c.h_min), c.h_max);
    }
    float4 p = st_pos[s];
    st_pos[s] = make_float4(p.x, p.y, p.z, hn);
}

// FP64 sums of 1/2 m v^2, m u, m v: per-block partials, then one ordered pass.
constexpr int RED_BLOCKS = 1024;
__global__ void k_energy_partials(int n, const float4 *__restrict__ vel, const float *__restrict__ mass,
                                  double *__restrict__ part) {
    __shared__ double sh[5][256];
    double a[5] = {0, 0, 0, 0, 0};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        float4 v = vel[s];
        double m = mass[s];
        double vx = v.x, vy = v.y, vz = v.z;
        a[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        a[1] += m * (double)v.w;
        a[2] += m * vx;
        a[3] += m * vy;
        a[4] += m * vz;
    }
    for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 5; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// the same sums per box: block b over the sorted slots of box b (box-major order)
__global__ void k_energy_box(const int32_t *__restrict__ start, const float4 *__restrict__ vel,
                             const float *__restrict__ mass, double *__restrict__ out) {
    __shared__ double sh[5][256];
    const int b = blockIdx.x;
    double a[5] = {0, 0, 0, 0, 0};
    for (int s = start[b] + threadIdx.x; s < start[b + 1]; s += blockDim.x) {
        float4 v = vel[s];
        double m = mass[s];
        double vx = v.x, vy = v.y, vz = v.z;
        a[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        a[1] += m * (double)v.w;
        a[2] += m * vx;
        a[3] += m * vy;
        a[4] += m * vz;
    }
    for (int k = 0; k < 5; k++) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 5; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[b * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_energy_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
    if (threadIdx.x < 5) {
        double s = 0;
        for (int b = 0; b < nb; b++) s += part[b * 8 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// h iteration: Thacker update of every particle not yet converged (eq:thacker)
__global__ void k_h_iter(int n, StepConsts c, float tol, const float *__restrict__ Nn, float *__restrict__ hs,
                         uint4 *__restrict__ q4, int32_t *__restrict__ flags, unsigned long long *notdone) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned nd = 0;
    if (s < n && !flags[s]) {
        float d = cbrtf(c.N_res / Nn[s]);
        float lam = d < 1.f ? 0.2f * (1.f + d * d) : 0.2f * (1.f + 1.f / (d * d * d));
        float hn = fminf(fmaxf(hs[s] * (1.f - lam + lam * d), c.h_min), c.h_max);
        // converged, or held at a bound that the update points beyond
        if (fabsf(d - 1.f) <= tol || hn == hs[s]) {
            flags[s] = 1;
        } else {
            hs[s] = hn;
            uint4 q = q4[s];
            q.w = to_fixed(hn);
            q4[s] = q;
            nd = 1;
        }
    }
    nd = __reduce_add_sync(0xffffffffu, nd);
    if ((threadIdx.x & 31) == 0 && nd) atomicAdd(notdone, (unsigned long long)nd);
}

// after the proposal wrote st_pos.w: the sorted h and the fixed-point support
__global__ void k_take_h(int n, const float4 *__restrict__ st_pos, float *__restrict__ hs, uint4 *__restrict__ q4) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float h = st_pos[s].w;
    hs[s] = h;
    q4[s].w = to_fixed(h);
}

__global__ void k_put_h(int n, const float *__restrict__ hs, float4 *__restrict__ st_pos) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    st_pos[s].w = hs[s];
}

// grad v records of the last evaluation into the new sorted order (new slot s
// takes old slot idx[s])
__global__ void k_permute_gv(int n, const int32_t *__restrict__ idx, const GvRec *__restrict__ in,
                             GvRec *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[s] = in[idx[s]];
}

__global__ void k_write_h(int n, const int32_t *__restrict__ perm, const float *__restrict__ hs, float4 *pos_h) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    pos_h[perm[s]].w = hs[s];
}

// ------------------------------------------------------------------ evaluation

// qV = (q, V) of every slot: after a P1 over some tiles only (time bins), the
// other slots keep their last V at their current position
__global__ void k_qv_refresh(int n, const uint4 *__restrict__ q4, const float *__restrict__ V, uint4 *__restrict__ qV) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint4 q = q4[s];
    qV[s] = make_uint4(q.x, q.y, q.z, __float_as_uint(V[s]));
}

// P1 -> P2 -> P3 -> P4 at the current build, with ctx->vel / ctx->mass set
// (over the tiles ctx->act only when that is set), then the per-particle
// time steps of every slot.
int evaluate(crk_ctx *ctx, cudaStream_t s) {
    int rc = run_volumes(ctx, s);
    if (!rc && ctx->act) {
        k_qv_refresh<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->q4, ctx->V, ctx->qV);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "pass records");
    }
    if (!rc) rc = run_corrections(ctx, true, s);
    if (!rc) rc = run_forces(ctx, s);
    if (rc) return rc;
    StepConsts c = step_consts(ctx->p);
    const bool batched = ctx->nbox > 1;
    unsigned long long *dtmin = batched ? ctx->box_dtmin : ctx->counters + CNT_DTMIN;
    const int nb = batched ? ctx->nbox : 1;
    k_fill_ull<<<grid_for(nb, 256), 256, 0, s>>>(nb, 0x7f7fffffull, dtmin);   // FLT_MAX bits
    k_cfl<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, c, ctx->hs, ctx->V, ctx->mass, ctx->vel, ctx->acc,
                                                  ctx->vq, ctx->gv, dtmin, batched ? ctx->sbox : nullptr,
                                                  ctx->d_dt, ctx->p.density ? ctx->rho : nullptr);
    ctx->launches += 2;
    CRK_LAUNCH_CHECK(ctx, "CFL");
    return CRK_OK;
}

}  // namespace crk

using namespace crk;

extern "C" int crk_reset_rates(crk_ctx *ctx) {
    if (!ctx) return CRK_EINVAL;
    ctx->rates_valid = 0;
    return CRK_OK;
}

// eq:hi solved at the drifted positions before the evaluation (h_mode >= 1):
// repeated P1 (summed in the walk, no lists) and eq:thacker updates of the
// particles not yet converged, the tile tree and tile-pair lists refitted to
// the new h after each (no re-sort), until every particle meets
// |Delta_N - 1| <= h_tol or sits at a bound its update points beyond (the
// rule of crk_h_iterate), or h_max_it passes.  h_mode 2 replaces the first
// update by the learned proposal (judged: particles already converged keep
// their h); its features take the grad v of the last evaluation, gv_old in the
// previous sorted order (idx: new slot -> old slot), and the step's dt.
// One eq:thacker update of every particle not yet converged (k_h_iter), then
// the tiles that still hold such a particle become ctx->act, so that the next
// P1 walks (and the next list rebuild covers) only those: a particle's count
// depends on its own h alone, so the others' counts stand.  Synchronises once;
// *nd = particles updated (0: all converged).
static int h_update(crk_ctx *ctx, const StepConsts &c, float tol, cudaStream_t s, unsigned long long *nd) {
    const int n = ctx->n;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_NOTDONE, 0, sizeof(unsigned long long), s));
    k_h_iter<<<grid_for(n, 256), 256, 0, s>>>(n, c, tol, ctx->Nn, ctx->hs, ctx->q4, ctx->flags,
                                              ctx->counters + CNT_NOTDONE);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "h iteration");
    int rc = unconverged_tiles(ctx, s);
    if (!rc) rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    *nd = ctx->h_counters[CNT_NOTDONE];
    ctx->nact = (int)ctx->h_counters[CNT_NACT];
    ctx->act = ctx->tact;
    return CRK_OK;
}

static int solve_h(crk_ctx *ctx, int n, const int32_t *idx, cudaStream_t s, int *iters, long long *unconv) {
    StepConsts c = step_consts(ctx->p);
    const float tol = ctx->p.h_tol;
    const int max_it = ctx->p.h_max_it;
    const int b = 256, g = grid_for(n, b);
    int rc = CRK_OK;
    if (ctx->p.h_mode == 2) {   // the last evaluation's grad v, in the new order (frec is free until P4)
        k_permute_gv<<<g, b, 0, s>>>(n, idx, ctx->gv, reinterpret_cast<GvRec *>(ctx->frec));
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "permute grad v");
    }
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * n, s));
    const int vo = ctx->volumes_only;
    ctx->volumes_only = 1;
    int it = 0;
    unsigned long long nd = 1;
    for (it = 1; it <= max_it; it++) {
        rc = run_volumes(ctx, s);
        if (rc) break;
        if (it == 1 && ctx->p.h_mode == 2) {
            double dt = 0.0;
            CRK_CUDA(ctx, cudaMemcpyAsync(&dt, ctx->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, s));
            CRK_CUDA(ctx, cudaStreamSynchronize(s));
            rc = propose_sorted(ctx, n, ctx->st_pos, reinterpret_cast<const GvRec *>(ctx->frec), ctx->Nn, (float)dt,
                                tol, s);
            if (rc) break;
            k_take_h<<<g, b, 0, s>>>(n, ctx->st_pos, ctx->hs, ctx->q4);
            ++ctx->launches;
            CRK_LAUNCH_CHECK(ctx, "proposed h");
            ctx->act = nullptr;   // every particle may have moved: the next pass walks all tiles
        } else {
            rc = h_update(ctx, c, tol, s, &nd);
            if (rc || nd == 0) break;
        }
        rc = build_tree(ctx, s);
        if (!rc) rc = rebuild_lists(ctx, s);
        if (!rc) rc = finish_build(ctx, s);
        if (rc) break;
    }
    const bool partial = ctx->act != nullptr;
    ctx->act = nullptr;
    ctx->nact = 0;
    ctx->volumes_only = vo;
    ctx->lists_valid = 0;
    if (!rc && partial) {   // the evaluation needs every tile's interaction list
        rc = rebuild_lists(ctx, s);
        if (!rc) rc = finish_build(ctx, s);
    }
    if (rc) return rc;
    *iters = it > max_it ? max_it : it;
    *unconv = (long long)nd;
    k_put_h<<<g, b, 0, s>>>(n, ctx->hs, ctx->st_pos);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "solved h");
    return CRK_OK;
}

// One KDK step of all boxes (one box unless batched).  dt_req applies to every
// box (<= 0: CFL); dt_box (device, one per box) overrides it when not null.
static int step_impl(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double dt_req,
                     const double *dt_box, bool batched, cudaStream_t s) {
    StepConsts c = step_consts(ctx->p);
    int rc;
    if (batched && ctx->p.h_mode != 0)
        return crk_set_error(ctx, CRK_ESTATE, "h_mode solves eq:hi in one-box steps only");
    int b = 256, g = grid_for(n, b);
    const bool fresh = !ctx->rates_valid || ctx->step_n != n || !ctx->built || ctx->n != n ||
                       (batched ? ctx->nbox < 1 : ctx->nbox > 1);
    if (fresh) {
        rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s, batched ? ctx->box_in : nullptr);
        if (!rc) rc = finish_build(ctx, s);
        if (rc) return rc;
        rc = gather_rows(ctx, pos_h, ctx->st_pos, 4, s);
        if (!rc) rc = gather_rows(ctx, vel_u, ctx->st_vel, 4, s);
        if (!rc) rc = gather_rows(ctx, mass, ctx->mass, 1, s);
        if (rc) return rc;
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->vel, ctx->st_vel, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        rc = evaluate(ctx, s);
        if (rc) return rc;
        ctx->rates_valid = 1;
        ctx->step_n = n;
    } else {
        rc = gather_rows(ctx, pos_h, ctx->st_pos, 4, s);
        if (!rc) rc = gather_rows(ctx, vel_u, ctx->st_vel, 4, s);
        if (rc) return rc;
    }
    const int nb = batched ? ctx->nbox : 1;
    const int32_t *sbox = batched ? ctx->sbox : nullptr;
    double *dtb = batched ? ctx->dtb : ctx->d_scalars;
    double *dtn = batched ? ctx->dtb_next : ctx->d_scalars + 16;   // the next step's dt
    if (fresh) CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_NEXT_OK, 0, 2 * sizeof(unsigned long long), s));
    k_pick_dt<<<grid_for(nb, 64), 64, 0, s>>>(nb, dt_req, dt_box, c.dt_max,
                                               batched ? ctx->box_dtmin : ctx->counters + CNT_DTMIN, dtb);
    k_next_check<<<1, 256, 0, s>>>(nb, dtb, dtn, ctx->counters);
    ctx->launches += 2;
    // first half kick with the cached rates, compatible energy of that kick
    // (formed ahead by the previous step's dual pass when its dt matches)
    k_kick1<<<g, b, 0, s>>>(n, dtb, sbox, ctx->st_vel, ctx->acc, ctx->vb, ctx->va);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "kick");
    rc = run_compatible(ctx, s, ctx->counters + CNT_SKIP);
    if (rc) return rc;
    k_take_next<<<g, b, 0, s>>>(n, ctx->counters, ctx->du_next, ctx->du);
    ++ctx->launches;
    k_half_drift<<<g, b, 0, s>>>(n, dtb, sbox, c, ctx->st_pos, ctx->st_vel, ctx->st_half, ctx->va, ctx->acc, ctx->du);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "drift");
    // rebuild at x1 (input order = current sorted order; boxes keep their particles)
    if (batched) CRK_CUDA(ctx, cudaMemcpyAsync(ctx->sbox_tmp, ctx->sbox, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    rc = build_cells_sorted(ctx, n, ctx->st_pos, ctx->perm, s, batched ? ctx->sbox_tmp : nullptr);
    if (!rc) rc = finish_build(ctx, s);
    if (rc) {
        ctx->rates_valid = 0;
        return rc;
    }
    k_permute3<<<g, b, 0, s>>>(n, ctx->idx_a, ctx->st_pos, ctx->st_tmp, ctx->st_vel, ctx->vb, ctx->st_half, ctx->va);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "permute state");
    float4 *t;
    t = ctx->st_pos; ctx->st_pos = ctx->st_tmp; ctx->st_tmp = t;
    t = ctx->st_vel; ctx->st_vel = ctx->vb; ctx->vb = t;
    t = ctx->st_half; ctx->st_half = ctx->va; ctx->va = t;
    rc = gather_rows(ctx, mass, ctx->mass, 1, s);
    if (rc) return rc;
    ctx->h_iters = 0;
    ctx->h_unconv = 0;
    if (ctx->p.h_mode >= 1) {   // eq:hi at x1 before the evaluation
        rc = solve_h(ctx, n, ctx->idx_a, s, &ctx->h_iters, &ctx->h_unconv);
        if (rc) {
            ctx->rates_valid = 0;
            return rc;
        }
    }
    // evaluation at (x1, p_p, u_p)
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->vel, ctx->st_vel, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    rc = evaluate(ctx, s);
    if (rc) {
        ctx->rates_valid = 0;
        return rc;
    }
    // second half kick and its compatible energy (the boxes' dt of this step;
    // the permutation kept every particle in its box)
    k_kick2<<<g, b, 0, s>>>(n, dtb, sbox, ctx->st_half, ctx->acc, ctx->vb, ctx->va);
    // the next step's dt under the same request, and both kicks' compatible
    // energy (this closing kick, the next opening kick) in one pass
    k_pick_dt<<<grid_for(nb, 64), 64, 0, s>>>(nb, dt_req, dt_box, c.dt_max,
                                               batched ? ctx->box_dtmin : ctx->counters + CNT_DTMIN, dtn);
    ctx->launches += 2;
    CRK_LAUNCH_CHECK(ctx, "kick");
    rc = run_compatible_dual(ctx, dtn, sbox, s);
    if (rc) return rc;
    k_set_next_ok<<<1, 1, 0, s>>>(ctx->counters);
    ++ctx->launches;
    k_finish<<<g, b, 0, s>>>(n, dtb, sbox, c, ctx->st_half, ctx->va, ctx->du, ctx->Nn, ctx->hs, ctx->st_vel,
                             ctx->st_pos);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "finish step");
    rc = scatter_rows(ctx, ctx->st_pos, pos_h, 4, s);
    if (!rc) rc = scatter_rows(ctx, ctx->st_vel, vel_u, 4, s);
    return rc;
}

extern "C" int crk_step(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double dt,
                        crk_diag *diag, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !vel_u || !mass) return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, false, s);
    if (rc || !diag) return rc;
    k_energy_partials<<<RED_BLOCKS, 256, 0, s>>>(n, ctx->st_vel, ctx->mass, ctx->d_red);
    ++ctx->launches;
    k_energy_final<<<1, 32, 0, s>>>(RED_BLOCKS, ctx->d_red, ctx->d_scalars + 2);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "diagnostics");
    double h[8];
    CRK_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, s));
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    diag->dt = h[0];
    diag->dt_next = (double)bits_to_float((uint32_t)ctx->h_counters[CNT_DTMIN]);
    diag->E_kin = h[2];
    diag->E_int = h[3];
    diag->P[0] = h[4];
    diag->P[1] = h[5];
    diag->P[2] = h[6];
    diag->pairs_gather = (long long)ctx->h_counters[CNT_PAIRS_G];
    diag->pairs_union = (long long)ctx->h_counters[CNT_PAIRS_U];
    diag->h_iterations = ctx->h_iters;
    diag->h_unconverged = ctx->h_unconv;
    return CRK_OK;
}

// The box table is loaded when it differs from the loaded one (and before the
// first batched step); loading forgets the rates.
static int reload_boxes_if_changed(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, cudaStream_t s) {
    bool same = ctx->nbox == nbox && nbox >= 1 && ctx->box_start && ctx->rates_valid && ctx->step_n == n;
    if (same) {
        std::vector<int32_t> cur((size_t)nbox + 1);
        CRK_CUDA(ctx, cudaMemcpyAsync(cur.data(), ctx->box_start, sizeof(int32_t) * ((size_t)nbox + 1),
                                      cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
        same = memcmp(cur.data(), box_start, sizeof(int32_t) * ((size_t)nbox + 1)) == 0;
    }
    if (same) return CRK_OK;
    ctx->rates_valid = 0;
    int rc = crk_ensure_particles(ctx, n);
    if (!rc) rc = load_boxes(ctx, n, nbox, box_start, s);
    return rc;
}

extern "C" int crk_step_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, float *pos_h,
                                float *vel_u, const float *mass, const double *dt, crk_diag *diag, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !vel_u || !mass || !box_start) return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = reload_boxes_if_changed(ctx, n, nbox, box_start, s);
    if (rc) return rc;
    const double *dt_box = nullptr;
    if (dt) {   // one requested step per box (<= 0: that box's CFL step)
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->box_red, dt, sizeof(double) * (size_t)nbox, cudaMemcpyHostToDevice, s));
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
        dt_box = ctx->box_red;
    }
    rc = step_impl(ctx, n, pos_h, vel_u, mass, 0.0, dt_box, nbox > 1, s);
    if (rc || !diag) return rc;
    const int nb = nbox;
    std::vector<double> red(8 * (size_t)nb), dts(nb);
    std::vector<unsigned long long> dtn(nb);
    if (nbox > 1) {
        k_energy_box<<<nb, 256, 0, s>>>(ctx->box_start, ctx->st_vel, ctx->mass, ctx->box_red);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "diagnostics");
        CRK_CUDA(ctx, cudaMemcpyAsync(red.data(), ctx->box_red, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaMemcpyAsync(dts.data(), ctx->dtb, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaMemcpyAsync(dtn.data(), ctx->box_dtmin, sizeof(unsigned long long) * nb,
                                      cudaMemcpyDeviceToHost, s));
    } else {
        k_energy_partials<<<RED_BLOCKS, 256, 0, s>>>(n, ctx->st_vel, ctx->mass, ctx->d_red);
        k_energy_final<<<1, 32, 0, s>>>(RED_BLOCKS, ctx->d_red, ctx->d_scalars + 2);
        ctx->launches += 2;
        CRK_LAUNCH_CHECK(ctx, "diagnostics");
        double h[8];
        CRK_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
        for (int k = 0; k < 5; k++) red[k] = h[2 + k];
        dts[0] = h[0];
    }
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    if (nbox == 1) dtn[0] = ctx->h_counters[CNT_DTMIN];
    for (int b = 0; b < nb; b++) {
        diag[b].dt = dts[b];
        diag[b].dt_next = (double)bits_to_float((uint32_t)dtn[b]);
        diag[b].E_kin = red[8 * b + 0];
        diag[b].E_int = red[8 * b + 1];
        diag[b].P[0] = red[8 * b + 2];
        diag[b].P[1] = red[8 * b + 3];
        diag[b].P[2] = red[8 * b + 4];
        diag[b].pairs_gather = (long long)ctx->h_counters[CNT_PAIRS_G];
        diag[b].pairs_union = (long long)ctx->h_counters[CNT_PAIRS_U];
        diag[b].h_iterations = 0;   // batched steps keep the evolved h
        diag[b].h_unconverged = 0;
    }
    return CRK_OK;
}

// ------------------------------------------------------------------ graphs

namespace {

// sticky overflow / invalid-input flag of a replayed step
__global__ void k_graph_check(unsigned long long *cnt, long long cap_ulist, int kcap) {
    if (cnt[CNT_ERR_INPUT] || cnt[CNT_PO_MISS] || cnt[CNT_TMA_ERR] || (long long)cnt[CNT_ULIST] > cap_ulist ||
        (long long)cnt[CNT_MAXCNT] > kcap)
        cnt[CNT_GRAPH_ERR] = 1ull;
}

void swap_state(crk_ctx *ctx) {   // the buffer rotation step_impl performs after its rebuild
    float4 *t;
    t = ctx->st_pos; ctx->st_pos = ctx->st_tmp; ctx->st_tmp = t;
    t = ctx->st_vel; ctx->st_vel = ctx->vb; ctx->vb = t;
    t = ctx->st_half; ctx->st_half = ctx->va; ctx->va = t;
}

unsigned long long fnv(unsigned long long h, unsigned long long v) {
    for (int k = 0; k < 8; k++) {
        h ^= (v >> (8 * k)) & 0xffull;
        h *= 1099511628211ull;
    }
    return h;
}

void drop_graphs(crk_ctx *ctx) {
    for (int k = 0; k < 2; k++) {
        if (ctx->gexec[k]) cudaGraphExecDestroy(ctx->gexec[k]);
        ctx->gexec[k] = nullptr;
        ctx->gkey[k] = 0;
    }
}

int run_diag(crk_ctx *ctx, int n, crk_diag *diag, cudaStream_t s) {
    k_energy_partials<<<RED_BLOCKS, 256, 0, s>>>(n, ctx->st_vel, ctx->mass, ctx->d_red);
    k_energy_final<<<1, 32, 0, s>>>(RED_BLOCKS, ctx->d_red, ctx->d_scalars + 2);
    ctx->launches += 2;
    CRK_LAUNCH_CHECK(ctx, "diagnostics");
    double h[8];
    CRK_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_scalars, sizeof(h), cudaMemcpyDeviceToHost, s));
    int rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    diag->dt = h[0];
    diag->dt_next = (double)bits_to_float((uint32_t)ctx->h_counters[CNT_DTMIN]);
    diag->E_kin = h[2];
    diag->E_int = h[3];
    diag->P[0] = h[4];
    diag->P[1] = h[5];
    diag->P[2] = h[6];
    diag->pairs_gather = (long long)ctx->h_counters[CNT_PAIRS_G];
    diag->pairs_union = (long long)ctx->h_counters[CNT_PAIRS_U];
    diag->h_iterations = ctx->h_iters;
    diag->h_unconverged = ctx->h_unconv;
    return CRK_OK;
}

}  // namespace

void crk::graph_free(crk_ctx *ctx) {
    drop_graphs(ctx);
    for (int k = 0; k < 2; k++)
        if (ctx->gev[k]) cudaEventDestroy(ctx->gev[k]);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->bk_pos) cudaFree(ctx->bk_pos);
    if (ctx->bk_vel) cudaFree(ctx->bk_vel);
    ctx->gstream = nullptr;
    ctx->bk_pos = ctx->bk_vel = nullptr;
    ctx->cap_bk = 0;
}

extern "C" int crk_set_expansion(crk_ctx *ctx, double a, double adot) {
    if (!ctx) return CRK_EINVAL;
    if (!(a > 0.0 && a < 1e30) || !(adot > -1e30 && adot < 1e30))
        return crk_set_error(ctx, CRK_EINVAL, "bad scale factor or rate");
    if (a != ctx->p.a || adot != ctx->p.adot) drop_graphs(ctx);   // graphs hold the old constants
    ctx->p.a = a;
    ctx->p.adot = adot;
    return CRK_OK;
}

extern "C" int crk_graph_stats(crk_ctx *ctx, long long *captures, long long *replays, long long *recoveries) {
    if (!ctx) return CRK_EINVAL;
    if (captures) *captures = ctx->gcaptures;
    if (replays) *replays = ctx->greplays;
    if (recoveries) *recoveries = ctx->grecoveries;
    return CRK_OK;
}

// Capture one steady-state step on the capture stream (kernels recorded, host
// logic run: the state buffers rotate as after the step).  Returns false when
// the step cannot be captured; the caller then steps eagerly.
static bool capture_step(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double dt, int p,
                         unsigned long long key, bool batched) {
    if (ctx->gexec[p]) cudaGraphExecDestroy(ctx->gexec[p]);
    ctx->gexec[p] = nullptr;
    ctx->gkey[p] = 0;
    int prof = ctx->prof_on;
    ctx->prof_on = 0;
    ctx->graph_mode = 1;
    cudaGraph_t graph = nullptr;
    int rc = 0;
    const long long l0 = ctx->launches;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, batched, ctx->gstream);
        if (!rc) {
            k_graph_check<<<1, 1, 0, ctx->gstream>>>(ctx->counters, ctx->cap_ulist, ctx->kcap);
            ++ctx->launches;
        }
        e = cudaStreamEndCapture(ctx->gstream, &graph);
    }
    ctx->graph_mode = 0;
    ctx->prof_on = prof;
    bool ok = !rc && e == cudaSuccess && graph &&
              cudaGraphInstantiate(&ctx->gexec[p], graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a failed capture leaves an error behind; the eager step reports its own
    if (!ok) {
        ctx->gexec[p] = nullptr;
        ctx->rates_valid = 0;   // the host logic ran, the kernels did not: start afresh
        return false;
    }
    ctx->gkey[p] = key;
    ctx->glaunch[p] = ctx->launches - l0;
    ctx->launches = l0;         // counted when the graph runs
    ctx->gcaptures++;
    return true;
}

static int steps_impl(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, int nsteps, double dt,
                      int use_graph, bool batched, cudaStream_t s) {
    int rc, done = 0;
    // eager steps: without graphs, from a fresh state (its first step sizes
    // every buffer a captured step uses) and while the passes are being tuned
    for (;;) {
        const bool fresh = !ctx->rates_valid || ctx->step_n != n || ctx->n != n || (ctx->nbox > 1) != batched;
        bool tuning = false;
        if (ctx->tune_on)
        {
            for (int k = PROF_P1; k <= PROF_P5; k++) tuning |= (k != PROF_PN && !ctx->tune_done[k]);
            tuning |= !ctx->tune_done[TUNE_P5_DUAL] || (ctx->p.density && !ctx->tune_done[PROF_DENS]);
        }
        // a step that solves eq:hi syncs the host once per iteration: never captured
        if (done == nsteps || (use_graph && !fresh && !tuning && ctx->p.h_mode == 0)) break;
        rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, batched, s);
        if (rc) return rc;
        done++;
    }
    if (done < nsteps) {
        // headroom for the replayed steps: list columns (they change only at a
        // walk, so one more eager step applies the new width) and tile-pair lists
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        const long long maxc = (long long)ctx->h_counters[CNT_MAXCNT];
        const long long nu = (long long)ctx->h_counters[CNT_ULIST];
        if (maxc + maxc / 2 > ctx->kcap && done < nsteps) {
            ctx->kcap = (int)((maxc + maxc / 2 + 31) / 32 * 32);
            rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, batched, s);
            if (rc) return rc;
            done++;
        }
        if (nu + nu / 2 > ctx->cap_ulist) {
            rc = crk_ensure_lists(ctx, 0, nu + nu / 2 + 1024);
            if (rc) return rc;
        }
    }
    if (done < nsteps) {
        // worst-case stored-force capacity (nothing grows inside a captured step;
        // the forces of the last evaluation are kept: the next kick reads them),
        // backup, capture stream
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
        rc = crk_grow_forces_keep(ctx, (long long)ctx->ntiles * ctx->kcap * 32);
        if (rc) return rc;
        if (ctx->p.pair_form == 1) {   // the pair-once arrays follow the tile lists' headroom
            rc = crk_ensure_pair_once(ctx);
            if (rc) return rc;
        }
        if (n > ctx->cap_bk) {
            if (ctx->bk_pos) cudaFree(ctx->bk_pos);
            if (ctx->bk_vel) cudaFree(ctx->bk_vel);
            ctx->bk_pos = ctx->bk_vel = nullptr;
            ctx->cap_bk = 0;
            CRK_CUDA(ctx, cudaMalloc((void **)&ctx->bk_pos, sizeof(float4) * (size_t)n));
            CRK_CUDA(ctx, cudaMalloc((void **)&ctx->bk_vel, sizeof(float4) * (size_t)n));
            ctx->cap_bk = n;
        }
        if (!ctx->gstream) {
            CRK_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
            CRK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
            CRK_CUDA(ctx, cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
        }
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->bk_pos, pos_h, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->bk_vel, vel_u, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_GRAPH_ERR, 0, sizeof(unsigned long long), s));
        CRK_CUDA(ctx, cudaEventRecord(ctx->gev[0], s));
        CRK_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
        bool eager = false;
        for (int k = done; k < nsteps; k++) {
            // which of the two buffer rotations the state is in
            const int p = (uintptr_t)ctx->st_pos < (uintptr_t)ctx->st_tmp ? 0 : 1;
            unsigned long long key = 1469598103934665603ull;
            unsigned long long dtbits;
            memcpy(&dtbits, &dt, sizeof(dtbits));
            const unsigned long long parts[] = {
                (unsigned long long)n, (unsigned long long)(uintptr_t)pos_h, (unsigned long long)(uintptr_t)vel_u,
                (unsigned long long)(uintptr_t)mass, ctx->alloc_gen, (unsigned long long)ctx->kcap,
                (unsigned long long)ctx->cap_ulist, (unsigned long long)(uintptr_t)ctx->st_pos, dtbits,
                (unsigned long long)batched * 7919ull + (unsigned long long)ctx->nbox};
            for (unsigned long long v : parts) key = fnv(key, v);
            const int tuned[] = {PROF_P1, PROF_P2, PROF_P3, PROF_P4, PROF_P5, TUNE_P5_DUAL, PROF_DENS};
            for (int t : tuned) key = fnv(key, (unsigned long long)(long long)ctx->tune_choice[t]);
            if (!eager && (!ctx->gexec[p] || ctx->gkey[p] != key)) {
                // capturing runs the step's host logic (its buffer rotation) but not its kernels
                if (!capture_step(ctx, n, pos_h, vel_u, mass, dt, p, key, batched)) eager = true;
            } else if (!eager) {
                swap_state(ctx);
            }
            if (eager) {   // capture unavailable: the remaining steps run eagerly on the capture stream
                rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, batched, ctx->gstream);
                if (rc) return rc;
                continue;
            }
            CRK_CUDA(ctx, cudaGraphLaunch(ctx->gexec[p], ctx->gstream));
            ctx->launches += ctx->glaunch[p];
            ctx->greplays++;
        }
        CRK_CUDA(ctx, cudaEventRecord(ctx->gev[1], ctx->gstream));
        CRK_CUDA(ctx, cudaStreamWaitEvent(s, ctx->gev[1], 0));
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        if (ctx->h_counters[CNT_GRAPH_ERR]) {
            // a replayed step outgrew a capacity despite the headroom: restore the
            // positions and velocities this run of replays started from and redo
            // its steps eagerly (their first step evaluates the rates afresh there)
            ctx->grecoveries++;
            CRK_CUDA(ctx, cudaMemcpyAsync(pos_h, ctx->bk_pos, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            CRK_CUDA(ctx, cudaMemcpyAsync(vel_u, ctx->bk_vel, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            drop_graphs(ctx);
            ctx->rates_valid = 0;
            for (int k = done; k < nsteps; k++) {
                rc = step_impl(ctx, n, pos_h, vel_u, mass, dt, nullptr, batched, s);
                if (rc) return rc;
            }
        }
    }
    return CRK_OK;
}

extern "C" int crk_steps(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, int nsteps,
                         double dt, int use_graph, crk_diag *diag, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !vel_u || !mass || nsteps < 0) return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    if (nsteps == 0) return CRK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = steps_impl(ctx, n, pos_h, vel_u, mass, nsteps, dt, use_graph, false, s);
    if (rc) return rc;
    return diag ? run_diag(ctx, n, diag, s) : CRK_OK;
}

extern "C" int crk_steps_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, float *pos_h,
                                 float *vel_u, const float *mass, int nsteps, double dt, int use_graph,
                                 void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !vel_u || !mass || !box_start || nsteps < 0)
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    if (nsteps == 0) return CRK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = reload_boxes_if_changed(ctx, n, nbox, box_start, s);
    if (rc) return rc;
    return steps_impl(ctx, n, pos_h, vel_u, mass, nsteps, dt, use_graph, nbox > 1, s);
}

static int h_iterate(crk_ctx *ctx, int n, float *pos_h, float tol, int max_it, int *iterations, cudaStream_t s);

// P1 is all the iteration needs: it runs as the fused volume walk, without
// per-particle neighbour lists or stored-force buffers.
extern "C" int crk_h_iterate(crk_ctx *ctx, int n, float *pos_h, float tol, int max_it, int *iterations,
                             void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !(tol > 0.f) || max_it < 1) return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    ctx->rates_valid = 0;
    int vo = ctx->volumes_only;
    ctx->volumes_only = 1;
    int rc = h_iterate(ctx, n, pos_h, tol, max_it, iterations, (cudaStream_t)stream);
    ctx->volumes_only = vo;
    ctx->lists_valid = 0;
    return rc;
}

static int h_iterate(crk_ctx *ctx, int n, float *pos_h, float tol, int max_it, int *iterations, cudaStream_t s) {
    int rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s);
    if (!rc) rc = finish_build(ctx, s);
    if (rc) return rc;
    StepConsts c = step_consts(ctx->p);
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * n, s));
    int it = 0;
    unsigned long long nd = 1;
    for (it = 1; it <= max_it; it++) {
        rc = run_volumes(ctx, s);
        if (!rc) rc = h_update(ctx, c, tol, s, &nd);
        if (rc || nd == 0) break;
        rc = build_tree(ctx, s);
        if (!rc) rc = rebuild_lists(ctx, s);
        if (!rc) rc = finish_build(ctx, s);
        if (rc) break;
    }
    ctx->act = nullptr;
    ctx->nact = 0;
    if (rc) return rc;
    if (iterations) *iterations = it > max_it ? max_it : it;
    k_write_h<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, ctx->hs, (float4 *)pos_h);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "write h");
    CRK_CUDA(ctx, cudaStreamSynchronize(s));
    if (nd) return crk_set_error(ctx, CRK_ENONCONV, "%llu particles not converged after %d iterations", nd, max_it);
    return CRK_OK;
}
