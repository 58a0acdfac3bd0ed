// crk_walk.cu -- per-particle neighbour lists, built once per evaluation from
// the tile interaction lists (CRK-HACC Sec. 2.3: interaction lists assembled
// once per hydro step and reused by every hydro kernel), and P1 volumes
// (Sec. 1.2 eq:vol, Sec. 2.6 eq:hi) over those lists.
//
// One walk: warp per i-tile over the pair-set tile list; every staged
// neighbour is tested once with the exact fixed-point predicate (integer work
// only).  Lane i writes its list into
// the tile's column layout with KCAP columns (entry column c of lane i at
// (tile * KCAP + c) * 32 + i): gather neighbours (j != i, |dq|^2 < H_i^2) from
// column 0 upwards with bit 31 = "j's kernel also reaches i", the other
// pair-set neighbours from column KCAP - 1 downwards.  A particle with more
// than KCAP neighbours sets the overflow maximum; the host then grows KCAP and
// walks again.  Stored pair forces use a compact layout: per-tile base (in
// units of 32 entries) from a scan of the per-tile maximum count.
#include "crk_pass.cuh"

namespace crk {

constexpr int WALK_WARPS = 8;

struct WalkArgs {
    int n, ntiles, kcap;
    const uint4 *q4;
    const float *hs;
    const uint2 *ofs;        // pair-set tile list per tile
    const uint32_t *tiles;
    const uint4 *tlo, *thi;  // tile boxes (xlo, ylo, zlo, Hmax), (xhi, yhi, zhi, count)
    float *V, *Nn;
    uint4 *qV;               // (qx, qy, qz, V bits)
    int32_t *cnt_g, *cnt_u;
    uint32_t *len_g, *len_u; // per-tile max counts
    unsigned long long *pairs_g, *pairs_u, *maxcnt;
    uint32_t *ent;
    const int32_t *sbox;     // batched boxes: box of each slot (BATCH only)
    const uint32_t *nbox;    // box range of each tile (BATCH only)
    const int32_t *act;      // may be null: walk the tiles act[0 .. ntiles) only
    int2 *lowc;              // may be null: per particle, gather and other entries with j < i
    unsigned long long *tests;   // lane tests of the exact predicate (LISTS walk)
};

// LISTS: write the lists; VOL: sum n_i in the walk (volumes-only contexts).
// circular distance (fixed point) from coordinate q to the arc [lo, hi]
// (which may wrap, lo > hi); differences modulo 2^32
__device__ __forceinline__ unsigned long long point_gap(uint32_t q, uint32_t lo, uint32_t hi) {
    if (q - lo <= hi - lo) return 0ull;
    uint32_t d1 = lo - q, d2 = q - hi;
    return (unsigned long long)(d1 < d2 ? d1 : d2);
}

// BATCH: the particles belong to independent boxes; j can be a neighbour of i
// only in i's box (the box ranges of tiles prune the rest).
template <bool LISTS, bool VOL, bool BATCH>
__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk(WalkArgs a) {
    __shared__ uint4 sq[WALK_WARPS][32];
    __shared__ int32_t sb[WALK_WARPS][BATCH ? 32 : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tw = blockIdx.x * WALK_WARPS + w;
    if (tw >= a.ntiles) return;
    const int tile = a.act ? a.act[tw] : tw;
    const int i = tile * TILE + lane;
    const bool valid = i < a.n;
    const uint4 qi = valid ? a.q4[i] : make_uint4(0, 0, 0, 0);
    const unsigned long long Hi2 = (unsigned long long)qi.w * qi.w;   // 0 for invalid lanes
    const float h = valid ? a.hs[i] : 1.f;
    const float inv_h = 1.f / h;
    const int kcap = a.kcap;
    uint32_t *const col0 = LISTS ? a.ent + (size_t)tile * kcap * 32 + lane : nullptr;
    float acc = 0.f;
    int cg = 0, co = 0;
    int lg = 0, lo_ = 0;   // entries with j < i: the candidate tiles come in ascending order
    uint32_t ntest = 0;    // kept staged particles (warp-uniform)
    const uint2 lo = a.ofs[tile];
    const uint4 Ilo = __ldg(a.tlo + tile), Ihi = __ldg(a.thi + tile);   // this tile's box, max H
    const int32_t bi = BATCH && valid ? a.sbox[i] : 0;
    const uint32_t Ib = BATCH ? __ldg(a.nbox + tile) : 0u;
    // software pipeline over the candidate tiles: the tile id two ahead, and
    // the box and this lane's staged particle of the next tile, are in flight
    // while the current tile is tested (each is otherwise a dependent L2 trip)
    const uint32_t *tl = a.tiles + lo.x;
    const int nt = (int)lo.y;
    int J1 = nt > 0 ? (int)__ldg(tl) : 0, J2 = nt > 1 ? (int)__ldg(tl + 1) : 0;
    uint4 lo1 = make_uint4(0, 0, 0, 0), hi1 = lo1, qn = lo1;
    if (nt > 0) {
        lo1 = __ldg(a.tlo + J1);
        hi1 = __ldg(a.thi + J1);
        if (J1 * TILE + lane < a.n) qn = __ldg(a.q4 + J1 * TILE + lane);
    }
    for (int t = 0; t < nt; t++) {
        const int J = J1;
        const uint4 Jlo = lo1, Jhi = hi1, qc = qn;
        J1 = J2;
        if (t + 2 < nt) J2 = (int)__ldg(tl + t + 2);
        if (t + 1 < nt) {
            lo1 = __ldg(a.tlo + J1);
            hi1 = __ldg(a.thi + J1);
            if (J1 * TILE + lane < a.n) qn = __ldg(a.q4 + J1 * TILE + lane);
        }
        // skip a neighbour tile that no lane's sphere (reach max(H_i, Hmax_J)) touches
        const unsigned long long gx = point_gap(qi.x, Jlo.x, Jhi.x), gy = point_gap(qi.y, Jlo.y, Jhi.y),
                                 gz = point_gap(qi.z, Jlo.z, Jhi.z);
        const unsigned long long reach = qi.w > Jlo.w ? qi.w : Jlo.w;
        bool near = valid && gx * gx + gy * gy + gz * gz < reach * reach;
        if constexpr (BATCH) {
            const uint32_t Jb = __ldg(a.nbox + J);
            near = near && (uint32_t)bi >= (Jb & 0xffffu) && (uint32_t)bi <= (Jb >> 16);
        }
        if (__ballot_sync(0xffffffffu, near) == 0u) continue;
        const int j0 = J * TILE;
        const int cnt = min(TILE, a.n - j0);
        // lane jj stages particle j0 + jj and keeps it only if it can be in the
        // pair set of some particle of this tile: its gap to the tile's box
        // below max(Hmax of the tile, H_j) (conservative, so the lists are
        // unchanged)
        __syncwarp();
        bool keep = false;
        if (lane < cnt) {
            const uint4 q = qc;
            sq[w][lane] = q;
            const unsigned long long hx = point_gap(q.x, Ilo.x, Ihi.x), hy = point_gap(q.y, Ilo.y, Ihi.y),
                                     hz = point_gap(q.z, Ilo.z, Ihi.z);
            const unsigned long long rj = q.w > Ilo.w ? q.w : Ilo.w;
            keep = hx * hx + hy * hy + hz * hz < rj * rj;
            if constexpr (BATCH) {
                const int32_t bj = __ldg(a.sbox + j0 + lane);
                sb[w][lane] = bj;
                keep = keep && (uint32_t)bj >= (Ib & 0xffffu) && (uint32_t)bj <= (Ib >> 16);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, keep);
        ntest += (uint32_t)__popc(mask);   // every lane tests every kept particle
        __syncwarp();
        // four staged particles per iteration: four independent predicate
        // chains in flight
        auto staged4 = [&](auto &&visit) {
            while (mask) {
                int jj[4];
                int cnt = 0;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    jj[u] = mask ? __ffs(mask) - 1 : jj[0];
                    if (mask) { mask &= mask - 1u; cnt++; }
                }
                uint4 qq[4];
                int dd[4][3];
                unsigned long long RR[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    qq[u] = sq[w][jj[u]];
                    dd[u][0] = (int)(qi.x - qq[u].x); dd[u][1] = (int)(qi.y - qq[u].y); dd[u][2] = (int)(qi.z - qq[u].z);
                    RR[u] = (BATCH && sb[w][jj[u]] != bi) ? ~0ull : r2_fixed(dd[u][0], dd[u][1], dd[u][2]);
                }
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u < cnt) visit(jj[u], qq[u], dd[u][0], dd[u][1], dd[u][2], RR[u]);
            }
        };
        if constexpr (LISTS) {
            // test phase: the exact predicate of every kept staged particle
            // sets this lane's bits (gather, other pair-set, "j reaches i");
            // write phase: each lane writes only its own entries, in staging
            // order, so the list-writing code runs once per entry rather than
            // once per staged particle
            unsigned gm = 0u, om = 0u, jm = 0u;
            staged4([&](int jj, const uint4 &qj, int, int, int, unsigned long long R2) {
                const bool in_i = R2 < Hi2;
                const bool in_j = R2 < (unsigned long long)qj.w * qj.w;
                const unsigned b = 1u << jj;
                gm |= in_i ? b : 0u;
                om |= (!in_i && in_j) ? b : 0u;
                jm |= in_j ? b : 0u;
            });
            if (!valid) gm = om = 0u;
            if (J == tile) {   // j != i
                gm &= ~(1u << lane);
                om &= ~(1u << lane);
            }
            if (J <= tile) {
                const unsigned below = J == tile ? lanemask_lt() : 0xffffffffu;
                lg = cg + __popc(gm & below);
                lo_ = co + __popc(om & below);
            }
            while (gm) {
                const int jj = __ffs(gm) - 1;
                gm &= gm - 1u;
                if (cg < kcap) col0[(size_t)cg * 32] = (uint32_t)(j0 + jj) | (((jm >> jj) & 1u) << 31);
                cg++;
            }
            while (om) {
                const int jj = __ffs(om) - 1;
                om &= om - 1u;
                if (co < kcap) col0[(size_t)(kcap - 1 - co) * 32] = (uint32_t)(j0 + jj);
                co++;
            }
        } else {
            staged4([&](int, const uint4 &, int dx, int dy, int dz, unsigned long long R2) {
                if (VOL && R2 < Hi2) {
                    Sep d = separation(dx, dy, dz);
                    float eta = d.r * inv_h;
                    float tt = fmaxf(1.f - eta, 0.f);
                    float t2 = tt * tt, t3 = t2 * tt;
                    acc = fmaf(t3 * t3, fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f), acc);
                }
            });
        }
    }
    const int cu = cg + co;
    if (valid) {
        if (VOL) {
            float ih3 = inv_h * inv_h * inv_h;
            float nsum = KW * ih3 * acc;                       // n_i, eq:vol
            a.V[i] = 1.f / nsum;
            if (a.Nn) a.Nn[i] = (K4PI_3 * h * h * h) * nsum;   // eq:hi
        }
        a.cnt_g[i] = cg;
        a.cnt_u[i] = cu;
        if (LISTS && a.lowc) a.lowc[i] = make_int2(lg, lo_);
    }
    uint32_t mg = __reduce_max_sync(0xffffffffu, (uint32_t)cg);
    uint32_t mu = __reduce_max_sync(0xffffffffu, (uint32_t)cu);
    uint32_t sg = __reduce_add_sync(0xffffffffu, (uint32_t)cg);
    uint32_t su = __reduce_add_sync(0xffffffffu, (uint32_t)cu);
    if (lane == 0) {
        a.len_g[tile] = min(mg, (uint32_t)kcap);
        a.len_u[tile] = min(mu, (uint32_t)kcap);
        atomicAdd(a.pairs_g, (unsigned long long)sg);
        atomicAdd(a.pairs_u, (unsigned long long)su);
        atomicMax(a.maxcnt, (unsigned long long)mu);
        if (LISTS) atomicAdd(a.tests, 32ull * ntest);
    }
}

// The walk for few tiles (time bins, act set): S warps share one tile, warp w
// testing the candidate tiles [w chunk, (w+1) chunk) of its list.  A first
// sweep counts every lane's gather and other neighbours per warp; their
// prefix over the warps gives each warp its columns, and a second sweep
// writes the entries there, so every list is exactly the one-warp walk's.
template <int S>
__global__ void __launch_bounds__(S * 32) k_walk_split(WalkArgs a) {
    __shared__ uint4 sq[S][32];
    __shared__ int cnt[2][S][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = a.act[blockIdx.x];
    const int i = tile * TILE + lane;
    const bool valid = i < a.n;
    const uint4 qi = valid ? a.q4[i] : make_uint4(0, 0, 0, 0);
    const unsigned long long Hi2 = (unsigned long long)qi.w * qi.w;
    const int kcap = a.kcap;
    uint32_t *const col0 = a.ent + (size_t)tile * kcap * 32 + lane;
    const uint2 lo = a.ofs[tile];
    const uint4 Ilo = __ldg(a.tlo + tile), Ihi = __ldg(a.thi + tile);
    const int nt = (int)lo.y;
    const int chunk = (nt + S - 1) / S;
    const int t0 = w * chunk, t1 = min(nt, t0 + chunk);
    int base_g = 0, base_o = 0, tot_g = 0, tot_o = 0;
    for (int phase = 0; phase < 2; phase++) {
        int cg = 0, co = 0;
        for (int t = t0; t < t1; t++) {
            const int J = (int)__ldg(a.tiles + lo.x + t);
            const uint4 Jlo = __ldg(a.tlo + J), Jhi = __ldg(a.thi + J);
            const unsigned long long gx = point_gap(qi.x, Jlo.x, Jhi.x), gy = point_gap(qi.y, Jlo.y, Jhi.y),
                                     gz = point_gap(qi.z, Jlo.z, Jhi.z);
            const unsigned long long reach = qi.w > Jlo.w ? qi.w : Jlo.w;
            const bool near = valid && gx * gx + gy * gy + gz * gz < reach * reach;
            if (__ballot_sync(0xffffffffu, near) == 0u) continue;
            const int j0 = J * TILE;
            const int cj = min(TILE, a.n - j0);
            __syncwarp();
            bool keep = false;
            if (lane < cj) {
                const uint4 q = __ldg(a.q4 + j0 + lane);
                sq[w][lane] = q;
                const unsigned long long hx = point_gap(q.x, Ilo.x, Ihi.x), hy = point_gap(q.y, Ilo.y, Ihi.y),
                                         hz = point_gap(q.z, Ilo.z, Ihi.z);
                const unsigned long long rj = q.w > Ilo.w ? q.w : Ilo.w;
                keep = hx * hx + hy * hy + hz * hz < rj * rj;
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            auto visit = [&](int jj, const uint4 &qj, unsigned long long R2) {
                const uint32_t j = (uint32_t)(j0 + jj);
                if (valid && (int)j != i) {
                    const bool in_i = R2 < Hi2;
                    const bool in_j = R2 < (unsigned long long)qj.w * qj.w;
                    if (in_i) {
                        const int c = base_g + cg;
                        if (phase == 1 && c < kcap) col0[(size_t)c * 32] = j | (in_j ? 0x80000000u : 0u);
                        cg++;
                    } else if (in_j) {
                        const int c = base_o + co;
                        if (phase == 1 && c < kcap) col0[(size_t)(kcap - 1 - c) * 32] = j;
                        co++;
                    }
                }
            };
            while (mask) {   // two staged neighbours per iteration, in staging order
                const int ja = __ffs(mask) - 1;
                mask &= mask - 1u;
                const bool two = mask != 0u;
                const int jb = two ? __ffs(mask) - 1 : ja;
                if (two) mask &= mask - 1u;
                const uint4 qa = sq[w][ja], qb = sq[w][jb];
                const unsigned long long Ra = r2_fixed((int)(qi.x - qa.x), (int)(qi.y - qa.y), (int)(qi.z - qa.z));
                const unsigned long long Rb = r2_fixed((int)(qi.x - qb.x), (int)(qi.y - qb.y), (int)(qi.z - qb.z));
                visit(ja, qa, Ra);
                if (two) visit(jb, qb, Rb);
            }
        }
        if (phase == 0) {
            cnt[0][w][lane] = cg;
            cnt[1][w][lane] = co;
            __syncthreads();
            for (int v = 0; v < S; v++) {
                if (v < w) {
                    base_g += cnt[0][v][lane];
                    base_o += cnt[1][v][lane];
                }
                tot_g += cnt[0][v][lane];
                tot_o += cnt[1][v][lane];
            }
        }
    }
    if (w != 0) return;
    const int cu = tot_g + tot_o;
    if (valid) {
        a.cnt_g[i] = tot_g;
        a.cnt_u[i] = cu;
    }
    uint32_t mg = __reduce_max_sync(0xffffffffu, (uint32_t)tot_g);
    uint32_t mu = __reduce_max_sync(0xffffffffu, (uint32_t)cu);
    uint32_t sg = __reduce_add_sync(0xffffffffu, (uint32_t)tot_g);
    uint32_t su = __reduce_add_sync(0xffffffffu, (uint32_t)cu);
    if (lane == 0) {
        a.len_g[tile] = min(mg, (uint32_t)kcap);
        a.len_u[tile] = min(mu, (uint32_t)kcap);
        atomicAdd(a.pairs_g, (unsigned long long)sg);
        atomicAdd(a.pairs_u, (unsigned long long)su);
        atomicMax(a.maxcnt, (unsigned long long)mu);
    }
}

// total stored-force units (32 entries each) = base[last] + len_u[last]
__global__ void k_total(int ntiles, const uint32_t *__restrict__ base, const uint32_t *__restrict__ len,
                        unsigned long long *out) {
    *out = ntiles ? (unsigned long long)base[ntiles - 1] + len[ntiles - 1] : 0ull;
}

static WalkArgs walk_args(crk_ctx *ctx) {
    WalkArgs a;
    a.n = ctx->n;
    a.ntiles = ctx->ntiles;
    a.kcap = ctx->kcap;
    a.q4 = ctx->q4;
    a.hs = ctx->hs;
    a.ofs = ctx->uofs;
    a.tiles = ctx->ulist;
    a.tlo = ctx->node_lo;
    a.thi = ctx->node_hi;
    a.V = ctx->V;
    a.Nn = ctx->Nn;
    a.qV = ctx->qV;
    a.cnt_g = ctx->cnt_g;
    a.cnt_u = ctx->cnt_u;
    a.len_g = ctx->len_g;
    a.len_u = ctx->len_u;
    a.pairs_g = ctx->counters + CNT_PAIRS_G;
    a.pairs_u = ctx->counters + CNT_PAIRS_U;
    a.maxcnt = ctx->counters + CNT_MAXCNT;
    a.ent = ctx->volumes_only ? nullptr : ctx->ent;
    a.sbox = ctx->nbox > 1 ? ctx->sbox : nullptr;
    a.nbox = ctx->nbox > 1 ? ctx->node_box : nullptr;
    a.act = ctx->act;
    if (ctx->act) a.ntiles = ctx->nact;
    a.lowc = ctx->volumes_only ? nullptr : ctx->lowc;
    a.tests = ctx->counters + CNT_WALK_TESTS;
    return a;
}

static int launch_walk(crk_ctx *ctx, cudaStream_t s) {
    if (!ctx->volumes_only) {
        int rc = crk_ensure_entries(ctx, (long long)ctx->ntiles * 32 * ctx->kcap, -1);
        if (rc) return rc;
    }
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_PAIRS_G, 0, 2 * sizeof(unsigned long long), s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_MAXCNT, 0, sizeof(unsigned long long), s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_WALK_TESTS, 0, sizeof(unsigned long long), s));
    if (ctx->act) {   // tiles left out of the walk take no list columns and no stored forces
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->len_g, 0, sizeof(uint32_t) * ctx->ntiles, s));
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->len_u, 0, sizeof(uint32_t) * ctx->ntiles, s));
        if (ctx->nact == 0) return CRK_OK;
    }
    prof_begin(ctx, PROF_LISTS, s);
    const int g = grid_for(ctx->act ? ctx->nact : ctx->ntiles, WALK_WARPS);
    const bool b = ctx->nbox > 1;
    const int nsm = ctx->nsm > 0 ? ctx->nsm : 152;
    if (ctx->act && !ctx->volumes_only && !b && ctx->nact < 8 * nsm)   // few tiles: 8 warps per tile
        k_walk_split<8><<<ctx->nact, 8 * 32, 0, s>>>(walk_args(ctx));
    else if (ctx->volumes_only && b)
        k_walk<false, true, true><<<g, WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    else if (ctx->volumes_only)
        k_walk<false, true, false><<<g, WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    else if (b)
        k_walk<true, false, true><<<g, WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    else
        k_walk<true, false, false><<<g, WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "neighbour walk");
    return CRK_OK;
}

// The walk and the list layout (synchronises once): on overflow grow KCAP and
// walk again; then lay out the stored pair forces.
int run_lists(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->lists_valid) return CRK_OK;
    if (ctx->volumes_only) return crk_set_error(ctx, CRK_ESTATE, "no neighbour lists in this context");
    if (ctx->n == 0) {
        ctx->lists_valid = 1;
        return CRK_OK;
    }
    int nt = ctx->ntiles;
    for (int attempt = 0; attempt < 3; attempt++) {
        int rc = launch_walk(ctx, s);
        if (rc) return rc;
        rc = scan_u32(ctx, ctx->len_u, ctx->tbase, nt, s);
        if (rc) return rc;
        k_total<<<1, 1, 0, s>>>(nt, ctx->tbase, ctx->len_u, ctx->counters + CNT_ENTRIES);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "list layout");
        if (ctx->graph_mode) {   // captured step: capacities were fixed beforehand, overflow checked after
            ctx->lists_valid = 1;
            return CRK_OK;
        }
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        long long maxc = (long long)ctx->h_counters[CNT_MAXCNT];
        if (maxc <= ctx->kcap) {
            long long units = (long long)ctx->h_counters[CNT_ENTRIES];
            rc = crk_ensure_entries(ctx, -1, units * 32);
            if (rc) return rc;
            ctx->entries = units * 32;
            ctx->lists_valid = 1;
            return CRK_OK;
        }
        ctx->kcap = (int)((maxc + maxc / 4 + 31) / 32 * 32);
    }
    return crk_set_error(ctx, CRK_ECAPACITY, "neighbour lists keep overflowing");
}

// The lists the passes walk, exported in caller order: thread per sorted slot
// s writes, from off[perm[s]], mode 0: its gather set (self first, then the
// front columns) as caller index | (j's kernel reaches i) << 31; mode 1: its
// pair set (front columns, then the back columns) as caller indices.
__global__ void k_export_lists(int n, int kcap, int mode, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ cnt_g, const int32_t *__restrict__ cnt_u,
                               const uint32_t *__restrict__ ent, const long long *__restrict__ off,
                               int32_t *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int tile = s / TILE, lane = s % TILE;
    const uint32_t *col0 = ent + (size_t)tile * kcap * 32 + lane;
    const int ci = perm[s];
    long long o = off[ci];
    const int cg = min(cnt_g[s], kcap), cu = min(cnt_u[s], kcap);
    if (mode == 0) out[o++] = (int32_t)((uint32_t)ci | 0x80000000u);
    for (int k = 0; k < cg; k++) {
        const uint32_t e = col0[(size_t)k * 32];
        const uint32_t j = (uint32_t)perm[e & 0x3fffffffu];
        out[o++] = (int32_t)(mode == 0 ? (j | (e & 0x80000000u)) : j);
    }
    if (mode == 1)
        for (int k = cg; k < cu; k++) out[o++] = perm[col0[(size_t)(kcap - 1 - (k - cg)) * 32] & 0x3fffffffu];
}

int run_export_lists(crk_ctx *ctx, int mode, const long long *off, int32_t *out, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    int rc = run_lists(ctx, s);
    if (rc) return rc;
    k_export_lists<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->kcap, mode, ctx->perm, ctx->cnt_g, ctx->cnt_u,
                                                          ctx->ent, off, out);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "export lists");
    return CRK_OK;
}

// P1 volumes over the gather lists (eq:vol, eq:hi), self included.
struct P1 {
    static constexpr bool GATHER = true;
    static constexpr int UNROLL = 4;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    using Rec = uint4;
    struct Params {
        const uint4 *q4;
        const float *hs;
        float *V, *Nn;
        uint4 *qV;
    };
    struct IState {
        uint4 q;
        float h, inv_h, acc;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        s.h = valid ? p.hs[i] : 1.f;
        s.inv_h = 1.f / s.h;
        s.acc = 1.f;                                   // self: W(0) / (495/(32 pi h^3)) = 1
    }
    __device__ static void zero(IState &s) { s.acc = 0.f; }
    __device__ static void merge(IState &s, const IState &o) { s.acc += o.acc; }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) { return __ldg(p.q4 + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &r, uint32_t, size_t, bool, const Params &) {
        int dx = (int)(s.q.x - r.x), dy = (int)(s.q.y - r.y), dz = (int)(s.q.z - r.z);
        Sep d = separation(dx, dy, dz);
        float eta = d.r * s.inv_h;
        float t = fmaxf(1.f - eta, 0.f);
        float t2 = t * t, t3 = t2 * t;
        s.acc = fmaf(t3 * t3, fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f), s.acc);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        float ih3 = s.inv_h * s.inv_h * s.inv_h;
        float nsum = KW * ih3 * s.acc;                       // n_i, eq:vol
        float V = 1.f / nsum;
        p.V[i] = V;
        if (p.Nn) p.Nn[i] = (K4PI_3 * s.h * s.h * s.h) * nsum;   // eq:hi
        p.qV[i] = make_uint4(s.q.x, s.q.y, s.q.z, __float_as_uint(V));
    }
};

// P1 volumes: the walk (if the lists are stale) and the list pass; a
// volumes-only context sums n_i inside the walk instead.
int run_volumes(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    if (ctx->volumes_only) {
        ctx->lists_valid = 0;
        return launch_walk(ctx, s);
    }
    int rc = run_lists(ctx, s);
    if (rc) return rc;
    P1::Params p{ctx->q4, ctx->hs, ctx->V, ctx->Nn, ctx->qV};
    return launch_lpass<P1, 8>(ctx, PROF_P1, p, s, "P1 volumes");
}

}  // namespace crk
