// crk_walk.cu -- per-particle neighbour lists, built once per evaluation from
// the tile interaction lists (CRK-HACC Sec. 2.3: interaction lists assembled
// once per hydro step and reused by every hydro kernel), with P1 volumes
// (Sec. 1.2 eq:vol, Sec. 2.6 eq:hi) fused into the counting walk.
//
// Walk 1 (count): warp per i-tile over the pair-set tile list; every staged
// neighbour is tested with the exact fixed-point predicate.  Lane i counts its
// gather neighbours (j != i, |dq|^2 < H_i^2) and its pair-set neighbours, and
// sums W(r, h_i) over gather(i) (self included) for n_i.
// Scan: tile capacities 32 * max_lane(pair-set count) -> tile base offsets.
// Walk 2 (fill): the same walk writes lane i's entries into the tile's column
// layout, entry k at base + 32 k + lane: first the gather neighbours (bit 31 =
// j's own kernel also reaches i), then the pair-set neighbours outside
// gather(i) (whose kernel always reaches i).  Both sections ascend in j.
#include "crk_pass.cuh"

namespace crk {

constexpr int WALK_WARPS = 8;

struct WalkArgs {
    int n, ntiles;
    const uint4 *q4;
    const float *hs;
    const uint2 *ofs;        // pair-set tile list per tile
    const uint32_t *tiles;
    // count outputs
    float *V, *Nn;
    uint4 *qV;               // (qx, qy, qz, V bits)
    int32_t *cnt_g, *cnt_u;
    uint32_t *len_g, *len_u; // per-tile max counts
    unsigned long long *pairs_g, *pairs_u;
    // fill
    const uint32_t *base;    // per-tile base offset (entries)
    uint32_t *ent;
};

template <bool FILL>
__global__ void __launch_bounds__(WALK_WARPS * 32) k_walk(WalkArgs a) {
    __shared__ uint4 sq[WALK_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * WALK_WARPS + w;
    if (tile >= a.ntiles) return;
    const int i = tile * TILE + lane;
    const bool valid = i < a.n;
    const uint4 qi = valid ? a.q4[i] : make_uint4(0, 0, 0, 0);
    const unsigned long long Hi2 = (unsigned long long)qi.w * qi.w;   // 0 for invalid lanes
    const float h = valid ? a.hs[i] : 1.f;
    const float inv_h = 1.f / h;
    float acc = 0.f;
    int cg = 0, cu = 0;
    uint32_t kg = 0, ko = 0, tb = 0;
    if (FILL) {
        tb = a.base[tile];
        ko = valid ? (uint32_t)a.cnt_g[i] : 0u;
    }
    const uint2 lo = a.ofs[tile];
    for (uint32_t t = 0; t < lo.y; t++) {
        const int J = (int)a.tiles[lo.x + t];
        const int j0 = J * TILE;
        const int cnt = min(TILE, a.n - j0);
        __syncwarp();
        if (lane < cnt) sq[w][lane] = a.q4[j0 + lane];
        __syncwarp();
        for (int jj = 0; jj < cnt; jj++) {
            const uint4 qj = sq[w][jj];
            const int dx = (int)(qi.x - qj.x), dy = (int)(qi.y - qj.y), dz = (int)(qi.z - qj.z);
            const unsigned long long R2 = r2_fixed(dx, dy, dz);
            const bool in_i = R2 < Hi2;
            const bool in_j = valid && R2 < (unsigned long long)qj.w * qj.w;
            const bool self = (j0 + jj) == i;
            if (!FILL) {
                if (in_i) {
                    Sep d = separation(dx, dy, dz);
                    float eta = d.r * inv_h;
                    float tt = fmaxf(1.f - eta, 0.f);
                    float t2 = tt * tt, t3 = t2 * tt;
                    acc = fmaf(t3 * t3, fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f), acc);
                }
                if (!self) {
                    cg += in_i;
                    cu += (in_i || in_j);
                }
            } else if (!self) {
                const uint32_t j = (uint32_t)(j0 + jj);
                if (in_i) {
                    a.ent[tb + kg * 32u + lane] = j | (in_j ? 0x80000000u : 0u);
                    kg++;
                } else if (in_j) {
                    a.ent[tb + ko * 32u + lane] = j;
                    ko++;
                }
            }
        }
    }
    if (!FILL) {
        if (valid) {
            float ih3 = inv_h * inv_h * inv_h;
            float nsum = KW * ih3 * acc;                       // n_i, eq:vol
            float V = 1.f / nsum;
            a.V[i] = V;
            if (a.Nn) a.Nn[i] = (4.18879020f * h * h * h) * nsum;   // eq:hi
            a.qV[i] = make_uint4(qi.x, qi.y, qi.z, __float_as_uint(V));
            a.cnt_g[i] = cg;
            a.cnt_u[i] = cu;
        }
        uint32_t mg = __reduce_max_sync(0xffffffffu, (uint32_t)cg);
        uint32_t mu = __reduce_max_sync(0xffffffffu, (uint32_t)cu);
        uint32_t sg = __reduce_add_sync(0xffffffffu, (uint32_t)cg);
        uint32_t su = __reduce_add_sync(0xffffffffu, (uint32_t)cu);
        if (lane == 0) {
            a.len_g[tile] = mg;
            a.len_u[tile] = mu;
            atomicAdd(a.pairs_g, (unsigned long long)sg);
            atomicAdd(a.pairs_u, (unsigned long long)su);
        }
    }
}

// tile capacity 32 * max pair-set count; exclusive scan done by the caller
__global__ void k_tile_cap(int ntiles, const uint32_t *__restrict__ len_u, uint32_t *__restrict__ cap) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) cap[t] = 32u * len_u[t];
}

// total entries = base[last] + cap[last]
__global__ void k_total(int ntiles, const uint32_t *__restrict__ base, const uint32_t *__restrict__ cap,
                        unsigned long long *out) {
    *out = ntiles ? (unsigned long long)base[ntiles - 1] + cap[ntiles - 1] : 0ull;
}

static WalkArgs walk_args(crk_ctx *ctx) {
    WalkArgs a;
    a.n = ctx->n;
    a.ntiles = ctx->ntiles;
    a.q4 = ctx->q4;
    a.hs = ctx->hs;
    a.ofs = ctx->uofs;
    a.tiles = ctx->ulist;
    a.V = ctx->V;
    a.Nn = ctx->Nn;
    a.qV = ctx->qV;
    a.cnt_g = ctx->cnt_g;
    a.cnt_u = ctx->cnt_u;
    a.len_g = ctx->len_g;
    a.len_u = ctx->len_u;
    a.pairs_g = ctx->counters + CNT_PAIRS_G;
    a.pairs_u = ctx->counters + CNT_PAIRS_U;
    a.base = ctx->tbase;
    a.ent = ctx->ent;
    return a;
}

// Walk 1: counts and P1 volumes.
int run_volumes(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_PAIRS_G, 0, 2 * sizeof(unsigned long long), s));
    prof_begin(ctx, PROF_P1, s);
    k_walk<false><<<grid_for(ctx->ntiles, WALK_WARPS), WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "P1 volumes (walk 1)");
    ctx->lists_valid = 0;
    return CRK_OK;
}

// Scan and walk 2: per-particle lists for the passes after P1.  Synchronises
// once to size the entry buffer.
int run_lists(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) {
        ctx->lists_valid = 1;
        return CRK_OK;
    }
    int nt = ctx->ntiles;
    prof_begin(ctx, PROF_LISTS, s);
    k_tile_cap<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->len_u, ctx->tcap);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "tile capacities");
    int rc = scan_u32(ctx, ctx->tcap, ctx->tbase, nt, s);
    if (rc) return rc;
    k_total<<<1, 1, 0, s>>>(nt, ctx->tbase, ctx->tcap, ctx->counters + CNT_ENTRIES);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "entry total");
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    long long total = (long long)ctx->h_counters[CNT_ENTRIES];
    rc = crk_ensure_entries(ctx, total);
    if (rc) return rc;
    k_walk<true><<<grid_for(nt, WALK_WARPS), WALK_WARPS * 32, 0, s>>>(walk_args(ctx));
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "neighbour lists (walk 2)");
    ctx->entries = total;
    ctx->lists_valid = 1;
    return CRK_OK;
}

}  // namespace crk
