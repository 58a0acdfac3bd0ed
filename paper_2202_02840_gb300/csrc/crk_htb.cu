// crk_htb.cu -- hierarchical power-of-two time bins of CRK-HACC Sec. 2.1 (the
// hydro subcycles of eq:Usubsub): per-particle criteria Delta y_hyd and
// Delta y_acc, leaf-level bins with the f_l limiter, parabolic streaming of
// passive leaves, and the KDK step of eq:verletOP with compatible energy
// (eq:compEng) for the leaves ending a step.
//
// The leaves are the 32-particle tiles of the sorted order at the cycle
// start; they keep their particles (and the engine its sorted order) until
// the cycle ends.  Per tile: level, start tick and length of its current
// step.  Per sorted slot: the state (x, h), the half-step velocity and
// energy (p_1/2, u_1/2), the acceleration of the last evaluation, and the
// energy rate of the opening kick.  Each tick at which some leaf ends a step
// streams every particle, refits the tile boxes and tree, and runs the walk,
// P1..P5 and the kicks over the active tiles only (the engine's active-tile
// mode); the passes read the passive particles' streamed positions and
// velocities and their last evaluated V, A, B, grad A, grad B, grad v.
#include "crk_internal.cuh"

#include <math.h>
#include <string.h>

#include <vector>

namespace crk {

constexpr int NO_LEVEL = -(1 << 20);   // 'no wake-up' (far below any level - f_l)
constexpr unsigned FULLM = 0xffffffffu;

struct HtbConsts {
    double tick;         // Delta / 2^L
    double Delta;
    int L, f_l;
    float N_res, h_min, h_max;
};

// smallest l in [0, L] with Delta / 2^l < dt (FP64; the scaling by 2^-l is
// exact); L + 1 when none is
__device__ __forceinline__ int particle_level(float dt, double Delta, int L) {
    const double d = (double)dt;
    for (int l = 0; l <= L; l++)
        if (ldexp(Delta, -l) < d) return l;
    return L + 1;
}

__device__ __forceinline__ bool tile_active(const int32_t *tt0, const int32_t *tlen, int T, int t) {
    return tt0[T] + tlen[T] == t;
}

// Required level of each listed tile (warp per tile) from the per-particle
// time steps; mid-cycle the tile may rise one level only at a tick aligned
// with its doubled step.  Writes the tentative level.
__global__ void k_htb_req(int count, const int32_t *__restrict__ act, int n, const float *__restrict__ dt,
                          HtbConsts c, int mid, int t, int32_t *__restrict__ tlev, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const int T = act ? act[w] : w;
    const int s = T * TILE + lane;
    int l = 0;
    if (s < n) l = particle_level(dt[s], c.Delta, c.L);
    const unsigned deep = __ballot_sync(FULLM, l > c.L);
    l = __reduce_max_sync(FULLM, min(l, c.L));
    if (lane == 0) {
        if (mid) {
            const int lo = tlev[T];
            const int base = (lo > 0 && (t % (2 << (c.L - lo))) == 0) ? lo - 1 : lo;
            l = max(l, base);
        }
        tlev[T] = l;
        if (deep) atomicAdd(cnt + CNT_UNRES, (unsigned long long)__popc(deep));
    }
}

// One limiter sweep over the listed tiles (warp per tile), in place:
// l_T = max(l_T, max_{J on T's interaction list} l_J - f_l).  Levels only
// rise, every tile is written by its own warp only, and a sweep that changes
// nothing leaves the least fixed point above the starting levels.
__global__ void k_htb_limit(int count, const int32_t *__restrict__ act, const uint2 *__restrict__ ofs,
                            const uint32_t *__restrict__ list, int f_l, int32_t *tlev,
                            unsigned long long *changed) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const int T = act ? act[w] : w;
    const uint2 o = ofs[T];
    int m = NO_LEVEL;
    for (uint32_t k = lane; k < o.y; k += 32) m = max(m, ((volatile int32_t *)tlev)[list[o.x + k]]);
    m = __reduce_max_sync(FULLM, m) - f_l;
    if (lane == 0 && m > tlev[T]) {
        tlev[T] = m;
        atomicAdd(changed, 1ull);
    }
}

// Every passive tile on an active tile's interaction list is raised to at
// least (active level - f_l).
__global__ void k_htb_wake(int count, const int32_t *__restrict__ act, const uint2 *__restrict__ ofs,
                           const uint32_t *__restrict__ list, const int32_t *__restrict__ tlev,
                           const int32_t *__restrict__ tt0, const int32_t *__restrict__ tlen, int t, int f_l,
                           int32_t *twake) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= count) return;
    const int T = act[w];
    const uint2 o = ofs[T];
    const int target = tlev[T] - f_l;
    for (uint32_t k = lane; k < o.y; k += 32) {
        const int J = (int)list[o.x + k];
        if (!tile_active(tt0, tlen, J, t) && target > tlev[J]) atomicMax(twake + J, target);
    }
}

// Apply the wake-ups (warp per tile): the raised tile's step now ends at the
// first tick after t that is a multiple of its new step, and its half kick
// p_1/2 = p0 + a len/2 (u alike) shrinks with the step, which keeps its
// streamed trajectory.  Clears the wake-up levels.
__global__ void k_htb_apply_wake(int ntiles, int n, HtbConsts c, int t, int32_t *tlev, const int32_t *tt0,
                                 int32_t *tlen, int32_t *twake, const float4 *__restrict__ acc,
                                 const float *__restrict__ du_open, float4 *st_half, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int T = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (T >= ntiles) return;
    const int wl = twake[T];
    if (wl <= tlev[T]) {
        if (lane == 0) twake[T] = NO_LEVEL;
        return;
    }
    const int Sn = 1 << (c.L - wl);
    const int te = (t / Sn + 1) * Sn;
    const int nl = te - tt0[T];
    const float hd = (float)(0.5 * (double)(tlen[T] - nl) * c.tick);
    const int s = T * TILE + lane;
    if (s < n) {
        const float4 a = acc[s];
        float4 p = st_half[s];
        p.x = fmaf(-hd, a.x, p.x);
        p.y = fmaf(-hd, a.y, p.y);
        p.z = fmaf(-hd, a.z, p.z);
        p.w = fmaf(-hd, du_open[s], p.w);
        st_half[s] = p;
    }
    __syncwarp();
    if (lane == 0) {
        tlen[T] = nl;
        tlev[T] = wl;
        twake[T] = NO_LEVEL;
        atomicAdd(cnt + CNT_WAKE, 1ull);
    }
}

// Stream every particle from tick t to t1 along v(t) = p_1/2 + a (t - t_mid):
// x += (t1 - t) tick (p_1/2 + a tick ((t + t1)/2 - t_mid)), periodic wrap;
// write the streamed velocity and energy at t1 (the evaluation state), the
// fixed-point records and h of the refit, and (at the cycle end) each
// particle's closing half-kick duration.
__global__ void k_htb_drift(int n, HtbConsts c, int t, int t1, const int32_t *__restrict__ tt0,
                            const int32_t *__restrict__ tlen, float4 *st_pos, const float4 *__restrict__ st_half,
                            const float4 *__restrict__ acc, const float *__restrict__ du_open,
                            float4 *__restrict__ vel, uint4 *__restrict__ q4, float *__restrict__ hs,
                            float *__restrict__ hc) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int T = s / TILE;
    const double tm = (double)tt0[T] + 0.5 * (double)tlen[T];
    const float c1 = (float)(c.tick * (0.5 * (double)(t + t1) - tm));
    const float c2 = (float)(c.tick * ((double)t1 - tm));
    const float w = (float)((double)(t1 - t) * c.tick);
    const float4 ph = st_half[s], a = acc[s];
    float4 p = st_pos[s];
    float x[3] = {fmaf(w, fmaf(c1, a.x, ph.x), p.x), fmaf(w, fmaf(c1, a.y, ph.y), p.y),
                  fmaf(w, fmaf(c1, a.z, ph.z), p.z)};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        x[k] -= floorf(x[k]);
        if (x[k] >= 1.f) x[k] = 0.f;
        if (x[k] < 0.f) x[k] = 0.f;
    }
    p = make_float4(x[0], x[1], x[2], p.w);
    st_pos[s] = p;
    vel[s] = make_float4(fmaf(c2, a.x, ph.x), fmaf(c2, a.y, ph.y), fmaf(c2, a.z, ph.z), fmaf(c2, du_open[s], ph.w));
    q4[s] = make_uint4(to_fixed(p.x), to_fixed(p.y), to_fixed(p.z), to_fixed(p.w));
    hs[s] = p.w;
    if (hc) hc[s] = (float)(0.5 * (double)tlen[T] * c.tick);
}

// fixed-point records and h of the state (refit without a sort)
__global__ void k_htb_records(int n, const float4 *__restrict__ st_pos, uint4 *__restrict__ q4, float *__restrict__ hs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float4 p = st_pos[s];
    q4[s] = make_uint4(to_fixed(p.x), to_fixed(p.y), to_fixed(p.z), to_fixed(p.w));
    hs[s] = p.w;
}

// closing kick of the active leaves: vb = p_1/2, va = p_1/2 + a len tick/2;
// every other particle enters the compatible energy unkicked, vb = va = v(t)
__global__ void k_htb_close(int n, HtbConsts c, int t, const int32_t *__restrict__ tt0,
                            const int32_t *__restrict__ tlen, const float4 *__restrict__ st_half,
                            const float4 *__restrict__ acc, const float4 *__restrict__ vel, float4 *__restrict__ vb,
                            float4 *__restrict__ va) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int T = s / TILE;
    if (tile_active(tt0, tlen, T, t)) {
        const float h = (float)(0.5 * (double)tlen[T] * c.tick);
        const float4 p = st_half[s], a = acc[s];
        vb[s] = make_float4(p.x, p.y, p.z, 0.f);
        va[s] = make_float4(fmaf(h, a.x, p.x), fmaf(h, a.y, p.y), fmaf(h, a.z, p.z), 0.f);
    } else {
        const float4 v = vel[s];
        vb[s] = make_float4(v.x, v.y, v.z, 0.f);
        va[s] = vb[s];
    }
}

// after the closing kick: (p1, u1 = u_1/2 + du len tick/2) into st_half, and
// h advanced by one eq:thacker update of this evaluation (clamped)
__global__ void k_htb_after_close(int n, HtbConsts c, int t, const int32_t *__restrict__ tt0,
                                  const int32_t *__restrict__ tlen, float4 *st_half, const float4 *__restrict__ va,
                                  const float *__restrict__ du, const float *__restrict__ Nn, float4 *st_pos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int T = s / TILE;
    if (!tile_active(tt0, tlen, T, t)) return;
    const float h = (float)(0.5 * (double)tlen[T] * c.tick);
    const float4 a = va[s];
    st_half[s] = make_float4(a.x, a.y, a.z, fmaf(h, du[s], st_half[s].w));
    const float d = cbrtf(c.N_res / Nn[s]);
    const float lam = d < 1.f ? 0.2f * (1.f + d * d) : 0.2f * (1.f + 1.f / (d * d * d));
    float4 p = st_pos[s];
    float hn = p.w * (1.f - lam + lam * d);
    p.w = fminf(fmaxf(hn, c.h_min), c.h_max);
    st_pos[s] = p;
}

// opening kick of the active leaves with their new step: vb = p1,
// va = p1 + a len' tick/2; the others as in k_htb_close
__global__ void k_htb_open(int n, HtbConsts c, int t, const int32_t *__restrict__ tlev,
                           const int32_t *__restrict__ tt0, const int32_t *__restrict__ tlen,
                           const float4 *__restrict__ st_half, const float4 *__restrict__ acc,
                           const float4 *__restrict__ vel, float4 *__restrict__ vb, float4 *__restrict__ va) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int T = s / TILE;
    if (tile_active(tt0, tlen, T, t)) {
        const float h = (float)(0.5 * (double)(1 << (c.L - tlev[T])) * c.tick);
        const float4 p = st_half[s], a = acc[s];
        vb[s] = make_float4(p.x, p.y, p.z, 0.f);
        va[s] = make_float4(fmaf(h, a.x, p.x), fmaf(h, a.y, p.y), fmaf(h, a.z, p.z), 0.f);
    } else {
        const float4 v = vel[s];
        vb[s] = make_float4(v.x, v.y, v.z, 0.f);
        va[s] = vb[s];
    }
}

// after the opening kick: (p_1/2, u_1/2 = u1 + du len' tick/2), and du is the
// energy rate the passive streaming of the new step uses
__global__ void k_htb_after_open(int n, HtbConsts c, int t, const int32_t *__restrict__ tlev,
                                 const int32_t *__restrict__ tt0, const int32_t *__restrict__ tlen, float4 *st_half,
                                 const float4 *__restrict__ va, const float *__restrict__ du,
                                 float *__restrict__ du_open) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int T = s / TILE;
    if (!tile_active(tt0, tlen, T, t)) return;
    const float h = (float)(0.5 * (double)(1 << (c.L - tlev[T])) * c.tick);
    const float4 a = va[s];
    const float r = du[s];
    st_half[s] = make_float4(a.x, a.y, a.z, fmaf(h, r, st_half[s].w));
    du_open[s] = r;
}

// the active leaves start their new step at t
__global__ void k_htb_set_steps(int ntiles, HtbConsts c, int t, const int32_t *__restrict__ tlev, int32_t *tt0,
                                int32_t *tlen) {
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= ntiles || !tile_active(tt0, tlen, T, t)) return;
    tt0[T] = t;
    tlen[T] = 1 << (c.L - tlev[T]);
}

// earliest step end over the tiles
__global__ void k_htb_tnext(int ntiles, const int32_t *__restrict__ tt0, const int32_t *__restrict__ tlen,
                            unsigned long long *cnt) {
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned e = T < ntiles ? (unsigned)(tt0[T] + tlen[T]) : 0xffffffffu;
    const unsigned m = __reduce_min_sync(FULLM, e);
    if ((threadIdx.x & 31) == 0) atomicMin(cnt + CNT_TNEXT, (unsigned long long)m);
}

__global__ void k_htb_flags(int ntiles, const int32_t *__restrict__ tt0, const int32_t *__restrict__ tlen, int t,
                            uint32_t *__restrict__ flag) {
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T < ntiles) flag[T] = tile_active(tt0, tlen, T, t) ? 1u : 0u;
}

// active tiles in ascending order, their count and their particles
__global__ void k_htb_compact(int ntiles, int n, const uint32_t *__restrict__ flag, const uint32_t *__restrict__ ofs,
                              int32_t *__restrict__ act, unsigned long long *cnt) {
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned parts = 0;
    if (T < ntiles && flag[T]) {
        act[ofs[T]] = T;
        parts = (unsigned)min(TILE, n - T * TILE);
    }
    parts = __reduce_add_sync(FULLM, parts);
    if ((threadIdx.x & 31) == 0 && parts) atomicAdd(cnt + CNT_NACT + 1, (unsigned long long)parts);
    if (T == ntiles - 1) cnt[CNT_NACT] = ofs[T] + flag[T];
}

// each slot takes its tile's level (for the caller's per-particle view)
__global__ void k_htb_slot_level(int n, const int32_t *__restrict__ tlev, int32_t *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = tlev[s / TILE];
}

// state of the new order after the end-of-cycle sort: slot s takes old slot idx[s]
__global__ void k_htb_permute(int n, const int32_t *__restrict__ idx, const float4 *__restrict__ a,
                              float4 *__restrict__ ao, const float4 *__restrict__ b, float4 *__restrict__ bo,
                              const float4 *__restrict__ c, float4 *__restrict__ co, const float *__restrict__ d,
                              float *__restrict__ dout) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int o = idx[s];
    ao[s] = a[o];
    bo[s] = b[o];
    co[s] = c[o];
    dout[s] = d[o];
}

// end of the cycle, every particle closes its step with its own duration:
// vb = p_1/2, va = p_1/2 + a hc
__global__ void k_htb_close_all(int n, const float *__restrict__ hc, const float4 *__restrict__ st_half,
                                const float4 *__restrict__ acc, float4 *__restrict__ vb, float4 *__restrict__ va) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float h = hc[s];
    const float4 p = st_half[s], a = acc[s];
    vb[s] = make_float4(p.x, p.y, p.z, 0.f);
    va[s] = make_float4(fmaf(h, a.x, p.x), fmaf(h, a.y, p.y), fmaf(h, a.z, p.z), 0.f);
}

__global__ void k_htb_finish_all(int n, HtbConsts c, const float *__restrict__ hc, const float4 *__restrict__ st_half,
                                 const float4 *__restrict__ va, const float *__restrict__ du,
                                 const float *__restrict__ Nn, float4 *__restrict__ st_vel, float4 *st_pos) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float4 a = va[s];
    st_vel[s] = make_float4(a.x, a.y, a.z, fmaf(hc[s], du[s], st_half[s].w));
    const float d = cbrtf(c.N_res / Nn[s]);
    const float lam = d < 1.f ? 0.2f * (1.f + d * d) : 0.2f * (1.f + 1.f / (d * d * d));
    float4 p = st_pos[s];
    float hn = p.w * (1.f - lam + lam * d);
    p.w = fminf(fmaxf(hn, c.h_min), c.h_max);
    st_pos[s] = p;
}

// ------------------------------------------------------------------ host side

static HtbConsts htb_consts(const crk_ctx *ctx, double Delta, int L, int f_l) {
    HtbConsts c;
    c.Delta = Delta;
    c.L = L;
    c.f_l = f_l;
    c.tick = ldexp(Delta, -L);
    c.N_res = (float)ctx->p.N_res;
    c.h_min = (float)ctx->p.h_min;
    c.h_max = (float)ctx->p.h_max;
    return c;
}

template <class T>
static int grow(crk_ctx *ctx, T **p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    CRK_CUDA(ctx, cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)));
    ++ctx->alloc_gen;
    return CRK_OK;
}

static int ensure_htb(crk_ctx *ctx) {
    const int nt = ctx->ntiles, n = ctx->n;
    int rc = CRK_OK;
    if (nt > ctx->cap_htb) {
        ctx->cap_htb = 0;
        rc = grow(ctx, &ctx->tlev, nt);
        if (!rc) rc = grow(ctx, &ctx->tt0, nt);
        if (!rc) rc = grow(ctx, &ctx->tlen, nt);
        if (!rc) rc = grow(ctx, &ctx->twake, nt);
        if (!rc) rc = grow(ctx, &ctx->tflag, nt);
        if (!rc) rc = grow(ctx, &ctx->tscan, nt);
        if (!rc) rc = grow(ctx, &ctx->tact, nt);
        if (rc) return rc;
        ctx->cap_htb = nt;
    }
    if (n > ctx->cap_htbp) {
        ctx->cap_htbp = 0;
        rc = grow(ctx, &ctx->du_open, n);
        if (!rc) rc = grow(ctx, &ctx->hc, n);
        if (rc) return rc;
        ctx->cap_htbp = n;
    }
    return CRK_OK;
}

// tile t holds a particle whose eq:hi solve is not yet done (flags[s] == 0)
__global__ void k_unconv_flags(int ntiles, int n, const int32_t *__restrict__ flags, uint32_t *__restrict__ tflag) {
    const int T = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (T >= ntiles) return;
    const int s = T * TILE + (int)(threadIdx.x & 31);
    const bool open = s < n && flags[s] == 0;
    const unsigned m = __ballot_sync(FULLM, open);
    if ((threadIdx.x & 31) == 0) tflag[T] = m != 0u;
}

// The tiles that hold a particle not yet converged (ctx->flags == 0), in tile
// order, into ctx->tact; their count lands in ctx->counters[CNT_NACT] (read
// after the caller's next sync).  The h solves walk only these tiles.
int unconverged_tiles(crk_ctx *ctx, cudaStream_t s) {
    int rc = ensure_htb(ctx);
    if (rc) return rc;
    const int nt = ctx->ntiles;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_NACT, 0, 2 * sizeof(unsigned long long), s));
    k_unconv_flags<<<grid_for((long long)nt * 32, 256), 256, 0, s>>>(nt, ctx->n, ctx->flags, ctx->tflag);
    ++ctx->launches;
    rc = scan_u32(ctx, ctx->tflag, ctx->tscan, nt, s);
    if (rc) return rc;
    k_htb_compact<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->n, ctx->tflag, ctx->tscan, ctx->tact, ctx->counters);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "unconverged tiles");
    return CRK_OK;
}

void htb_free(crk_ctx *ctx) {
    int32_t **ti[] = {&ctx->tlev, &ctx->tt0, &ctx->tlen, &ctx->twake, &ctx->tact};
    for (auto p : ti)
        if (*p) { cudaFree(*p); *p = nullptr; }
    if (ctx->tflag) cudaFree(ctx->tflag);
    if (ctx->tscan) cudaFree(ctx->tscan);
    if (ctx->du_open) cudaFree(ctx->du_open);
    if (ctx->hc) cudaFree(ctx->hc);
    ctx->tflag = ctx->tscan = nullptr;
    ctx->du_open = ctx->hc = nullptr;
    ctx->cap_htb = ctx->cap_htbp = 0;
}

// Tile boxes, tree and tile interaction lists of the current records (all
// tiles, or ctx->act), growing the list buffer when it overflows.  The
// per-particle neighbour lists and stored forces are left as they are.
static int refit_lists(crk_ctx *ctx, cudaStream_t s) {
    const int keep = ctx->lists_valid;
    int rc = build_tree(ctx, s);
    if (!rc) rc = rebuild_lists(ctx, s);
    if (!rc) rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    long long nu = (long long)ctx->h_counters[CNT_ULIST];
    if (nu > ctx->cap_ulist) {
        rc = crk_ensure_lists(ctx, 0, nu + nu / 4 + 1024);
        if (!rc) rc = rebuild_lists(ctx, s);
        if (!rc) rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        if ((long long)ctx->h_counters[CNT_ULIST] > ctx->cap_ulist)
            return crk_set_error(ctx, CRK_ECAPACITY, "interaction lists overflow after growth");
    }
    ctx->lists_valid = keep;
    return CRK_OK;
}

// Limiter sweeps over all tiles (act null) or the listed ones until a sweep
// raises nothing.  Every sweep that changes something raises some level by
// at least one, so ntiles (L + 1) + 1 sweeps always suffice.
static int limit(crk_ctx *ctx, const int32_t *act, int count, int f_l, int L, cudaStream_t s) {
    if (count == 0) return CRK_OK;
    const long long cap = (long long)ctx->ntiles * (L + 1) + 2;
    for (long long it = 0; it < cap; it += 4) {
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_CHANGED, 0, sizeof(unsigned long long), s));
        for (int k = 0; k < 4; k++) {
            k_htb_limit<<<grid_for((long long)count * 32, 256), 256, 0, s>>>(count, act, ctx->uofs, ctx->ulist, f_l,
                                                                         ctx->tlev, ctx->counters + CNT_CHANGED);
            ++ctx->launches;
        }
        CRK_LAUNCH_CHECK(ctx, "level limiter");
        int rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        if (ctx->h_counters[CNT_CHANGED] == 0) return CRK_OK;
    }
    return crk_set_error(ctx, CRK_ENONCONV, "level limiter did not converge");
}

// earliest step end, and the active list of that tick (synchronises)
static int next_tick(crk_ctx *ctx, int *t_next, cudaStream_t s) {
    const int nt = ctx->ntiles;
    const unsigned long long big = 0xffffffffull;
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->counters + CNT_TNEXT, &big, sizeof(big), cudaMemcpyHostToDevice, s));
    k_htb_tnext<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->tt0, ctx->tlen, ctx->counters);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "next tick");
    int rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    *t_next = (int)ctx->h_counters[CNT_TNEXT];
    return CRK_OK;
}

static int active_list(crk_ctx *ctx, int t, long long *parts, cudaStream_t s) {
    const int nt = ctx->ntiles;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_NACT, 0, 2 * sizeof(unsigned long long), s));
    k_htb_flags<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->tt0, ctx->tlen, t, ctx->tflag);
    ++ctx->launches;
    int rc = scan_u32(ctx, ctx->tflag, ctx->tscan, nt, s);
    if (rc) return rc;
    k_htb_compact<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->n, ctx->tflag, ctx->tscan, ctx->tact, ctx->counters);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "active leaves");
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    ctx->nact = (int)ctx->h_counters[CNT_NACT];
    *parts = (long long)ctx->h_counters[CNT_NACT + 1];
    return CRK_OK;
}

static void leave_active_mode(crk_ctx *ctx) {
    ctx->act = nullptr;
    ctx->nact = 0;
}

static int cycle_impl(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, const HtbConsts &c,
                      crk_htb_stats *st, cudaStream_t s) {
    int rc;
    const int b = 256, g = grid_for(n, b);
    const bool fresh = !ctx->rates_valid || ctx->step_n != n || !ctx->built || ctx->n != n || ctx->nbox > 1;
    if (fresh) {
        rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s);
        if (!rc) rc = finish_build(ctx, s);
        if (!rc) rc = gather_rows(ctx, pos_h, ctx->st_pos, 4, s);
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
    ctx->rates_valid = 0;   // until the cycle completes
    rc = ensure_htb(ctx);
    if (rc) return rc;
    const int nt = ctx->ntiles;
    // leaf boxes and interaction lists at the state (current h)
    k_htb_records<<<g, b, 0, s>>>(n, ctx->st_pos, ctx->q4, ctx->hs);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "leaf records");
    rc = refit_lists(ctx, s);
    if (rc) return rc;
    // levels at the cycle start: requirement, then the limiter's fixed point
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_UNRES, 0, 2 * sizeof(unsigned long long), s));
    k_htb_req<<<grid_for((long long)nt * 32, 256), 256, 0, s>>>(nt, nullptr, n, ctx->d_dt, c, 0, 0, ctx->tlev,
                                                              ctx->counters);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "leaf levels");
    rc = limit(ctx, nullptr, nt, c.f_l, c.L, s);
    if (rc) return rc;
    if (st) {
        std::vector<int32_t> lev(nt);
        CRK_CUDA(ctx, cudaMemcpyAsync(lev.data(), ctx->tlev, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
        memset(st->level_count, 0, sizeof(st->level_count));
        for (int v : lev) st->level_count[v < 0 ? 0 : (v > 31 ? 31 : v)]++;
        st->leaves = nt;
    }
    // every leaf opens its first step at tick 0 (t0 = len = 0 marks it active)
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->tt0, 0, sizeof(int32_t) * nt, s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->tlen, 0, sizeof(int32_t) * nt, s));
    std::vector<int32_t> none(nt, NO_LEVEL);
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->twake, none.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->st_half, ctx->st_vel, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    k_htb_open<<<g, b, 0, s>>>(n, c, 0, ctx->tlev, ctx->tt0, ctx->tlen, ctx->st_half, ctx->acc, ctx->vel, ctx->vb,
                               ctx->va);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "opening kick");
    rc = run_compatible(ctx, s);
    if (rc) return rc;
    k_htb_after_open<<<g, b, 0, s>>>(n, c, 0, ctx->tlev, ctx->tt0, ctx->tlen, ctx->st_half, ctx->va, ctx->du,
                                     ctx->du_open);
    k_htb_set_steps<<<grid_for(nt, 256), 256, 0, s>>>(nt, c, 0, ctx->tlev, ctx->tt0, ctx->tlen);
    ctx->launches += 2;
    CRK_LAUNCH_CHECK(ctx, "opening kick");
    long long evals = 0;
    int ticks = 0;
    const int T = 1 << c.L;
    int t = 0;
    for (;;) {
        int t1;
        rc = next_tick(ctx, &t1, s);
        if (rc) return rc;
        if (t1 <= t || t1 > T) return crk_set_error(ctx, CRK_ESTATE, "time bins: bad next tick %d after %d", t1, t);
        ++ticks;
        if (t1 == T) {
            k_htb_drift<<<g, b, 0, s>>>(n, c, t, t1, ctx->tt0, ctx->tlen, ctx->st_pos, ctx->st_half, ctx->acc,
                                        ctx->du_open, ctx->vel, ctx->q4, ctx->hs, ctx->hc);
            ++ctx->launches;
            CRK_LAUNCH_CHECK(ctx, "stream");
            break;
        }
        long long parts = 0;
        rc = active_list(ctx, t1, &parts, s);
        if (rc) return rc;
        evals += parts;
        k_htb_drift<<<g, b, 0, s>>>(n, c, t, t1, ctx->tt0, ctx->tlen, ctx->st_pos, ctx->st_half, ctx->acc,
                                    ctx->du_open, ctx->vel, ctx->q4, ctx->hs, nullptr);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "stream");
        t = t1;
        ctx->act = ctx->tact;
        rc = refit_lists(ctx, s);
        if (!rc) {
            ctx->lists_valid = 0;
            rc = evaluate(ctx, s);
        }
        if (rc) {
            leave_active_mode(ctx);
            return rc;
        }
        // closing kick, its compatible energy, h
        k_htb_close<<<g, b, 0, s>>>(n, c, t, ctx->tt0, ctx->tlen, ctx->st_half, ctx->acc, ctx->vel, ctx->vb, ctx->va);
        ++ctx->launches;
        rc = run_compatible(ctx, s);
        if (rc) {
            leave_active_mode(ctx);
            return rc;
        }
        k_htb_after_close<<<g, b, 0, s>>>(n, c, t, ctx->tt0, ctx->tlen, ctx->st_half, ctx->va, ctx->du, ctx->Nn,
                                          ctx->st_pos);
        // new levels of the active leaves, limiter over them, wake-ups
        k_htb_req<<<grid_for((long long)ctx->nact * 32, 256), 256, 0, s>>>(ctx->nact, ctx->tact, n, ctx->d_dt, c, 1,
                                                                           t, ctx->tlev, ctx->counters);
        ctx->launches += 2;
        CRK_LAUNCH_CHECK(ctx, "leaf levels");
        rc = limit(ctx, ctx->tact, ctx->nact, c.f_l, c.L, s);
        if (rc) {
            leave_active_mode(ctx);
            return rc;
        }
        k_htb_wake<<<grid_for((long long)ctx->nact * 32, 256), 256, 0, s>>>(ctx->nact, ctx->tact, ctx->uofs,
                                                                            ctx->ulist, ctx->tlev, ctx->tt0,
                                                                            ctx->tlen, t, c.f_l, ctx->twake);
        k_htb_apply_wake<<<grid_for((long long)nt * 32, 256), 256, 0, s>>>(nt, n, c, t, ctx->tlev, ctx->tt0,
                                                                           ctx->tlen, ctx->twake, ctx->acc,
                                                                           ctx->du_open, ctx->st_half,
                                                                           ctx->counters);
        // opening kick of the new step
        k_htb_open<<<g, b, 0, s>>>(n, c, t, ctx->tlev, ctx->tt0, ctx->tlen, ctx->st_half, ctx->acc, ctx->vel,
                                   ctx->vb, ctx->va);
        ctx->launches += 3;
        CRK_LAUNCH_CHECK(ctx, "wake-ups and opening kick");
        rc = run_compatible(ctx, s);
        leave_active_mode(ctx);
        if (rc) return rc;
        k_htb_after_open<<<g, b, 0, s>>>(n, c, t, ctx->tlev, ctx->tt0, ctx->tlen, ctx->st_half, ctx->va, ctx->du,
                                         ctx->du_open);
        k_htb_set_steps<<<grid_for(nt, 256), 256, 0, s>>>(nt, c, t, ctx->tlev, ctx->tt0, ctx->tlen);
        ctx->launches += 2;
        CRK_LAUNCH_CHECK(ctx, "opening kick");
    }
    // end of the cycle: every leaf ends its step; sort again, evaluate all,
    // close every step with its own duration
    rc = build_cells_sorted(ctx, n, ctx->st_pos, ctx->perm, s);
    if (!rc) rc = finish_build(ctx, s);
    if (rc) return rc;
    k_htb_permute<<<g, b, 0, s>>>(n, ctx->idx_a, ctx->st_pos, ctx->st_tmp, ctx->vel, ctx->vb, ctx->st_half, ctx->va,
                                  ctx->hc, ctx->st_tmp1);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "permute state");
    float4 *tp;
    tp = ctx->st_pos; ctx->st_pos = ctx->st_tmp; ctx->st_tmp = tp;
    tp = ctx->vel; ctx->vel = ctx->vb; ctx->vb = tp;
    tp = ctx->st_half; ctx->st_half = ctx->va; ctx->va = tp;
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->hc, ctx->st_tmp1, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    rc = gather_rows(ctx, mass, ctx->mass, 1, s);
    if (!rc) rc = evaluate(ctx, s);
    if (rc) return rc;
    evals += n;
    k_htb_close_all<<<g, b, 0, s>>>(n, ctx->hc, ctx->st_half, ctx->acc, ctx->vb, ctx->va);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "closing kick");
    rc = run_compatible(ctx, s);
    if (rc) return rc;
    k_htb_finish_all<<<g, b, 0, s>>>(n, c, ctx->hc, ctx->st_half, ctx->va, ctx->du, ctx->Nn, ctx->st_vel, ctx->st_pos);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "finish cycle");
    rc = scatter_rows(ctx, ctx->st_pos, pos_h, 4, s);
    if (!rc) rc = scatter_rows(ctx, ctx->st_vel, vel_u, 4, s);
    if (!rc) CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_NEXT_OK, 0, sizeof(unsigned long long), s));
    if (!rc) rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    ctx->rates_valid = 1;
    ctx->step_n = n;
    if (st) {
        st->ticks = ticks;
        st->evaluations = evals;
        st->wakeups = (long long)ctx->h_counters[CNT_WAKE];
        st->unresolved = (long long)ctx->h_counters[CNT_UNRES];
    }
    return CRK_OK;
}

}  // namespace crk

using namespace crk;

extern "C" int crk_cycle(crk_ctx *ctx, int n, float *pos_h, float *vel_u, const float *mass, double Delta, int L,
                         int f_l, crk_htb_stats *stats, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !vel_u || !mass || !(Delta > 0.0) || !isfinite(Delta) || L < 0 || L > 20 || f_l < 0)
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    if (ctx->nbox > 1) return crk_set_error(ctx, CRK_ESTATE, "time bins cover one box");
    if (ctx->p.a != 1.0 || ctx->p.adot != 0.0 || ctx->p.density != 0)
        return crk_set_error(ctx, CRK_EINVAL, "time bins are built for a static box (a = 1, adot = 0) and rho = m/V");
    if (ctx->volumes_only) return crk_set_error(ctx, CRK_ESTATE, "no neighbour lists in this context");
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = cycle_impl(ctx, n, pos_h, vel_u, mass, htb_consts(ctx, Delta, L, f_l), stats, s);
    leave_active_mode(ctx);
    if (rc) ctx->rates_valid = 0;
    return rc;
}

extern "C" int crk_htb_levels(crk_ctx *ctx, int n, const float *pos_h, const float *dt, double Delta, int L, int f_l,
                              int32_t *level, long long *unresolved, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n <= 0 || !pos_h || !dt || !level || !(Delta > 0.0) || !isfinite(Delta) || L < 0 || L > 20 || f_l < 0)
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    leave_active_mode(ctx);
    int rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s);
    if (!rc) rc = finish_build(ctx, s);
    if (!rc) rc = ensure_htb(ctx);
    if (!rc) rc = gather_rows(ctx, dt, ctx->d_dt, 1, s);
    if (rc) return rc;
    ctx->rates_valid = 0;
    const HtbConsts c = htb_consts(ctx, Delta, L, f_l);
    const int nt = ctx->ntiles;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_UNRES, 0, sizeof(unsigned long long), s));
    k_htb_req<<<grid_for((long long)nt * 32, 256), 256, 0, s>>>(nt, nullptr, n, ctx->d_dt, c, 0, 0, ctx->tlev,
                                                              ctx->counters);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "leaf levels");
    rc = limit(ctx, nullptr, nt, f_l, L, s);
    if (rc) return rc;
    k_htb_slot_level<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->tlev, reinterpret_cast<int32_t *>(ctx->st_tmp1));
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "leaf levels");
    rc = scatter_rows(ctx, ctx->st_tmp1, level, 1, s);
    if (!rc) rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    if (unresolved) *unresolved = (long long)ctx->h_counters[CNT_UNRES];
    return CRK_OK;
}
