// crk_pass.cuh -- warp-per-tile skeleton of the pair passes.
//
// One warp owns one i-tile (lane = particle i of 32 consecutive sorted
// particles) and walks the tile's interaction list.  Each neighbour tile J is
// staged once in shared memory (lane l loads record J*32+l, coalesced) and
// every lane then loops over the 32 staged records, testing the exact
// fixed-point predicate and accumulating in registers.  No atomics, no
// inter-warp synchronisation: results are deterministic.
#pragma once

#include "crk_internal.cuh"

#include <type_traits>

namespace crk {

struct PassGeom {
    int n;
    int ntiles;
    const uint2 *ofs;        // per i-tile (offset, count) into list
    const uint32_t *list;    // neighbour tile ids
    unsigned long long *pairs;  // optional pair counter
};

// P must provide: Params, JRec, IState,
//   init(IState&, int i, bool valid, const Params&)
//   stage(JRec&, int j, const Params&)
//   pair(IState&, const JRec&, int j, int i, bool valid, const Params&)
//   finish(IState&, int i, const Params&)           (valid lanes only)
//   count(const IState&) -> pairs of this lane
template <class P, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_pass(PassGeom g, typename P::Params prm) {
    __shared__ typename P::JRec sj[WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * WARPS + w;
    if (tile >= g.ntiles) return;
    const int i = tile * TILE + lane;
    const bool valid = i < g.n;
    typename P::IState st;
    P::init(st, i, valid, prm);
    const uint2 lo = g.ofs[tile];
    for (uint32_t t = 0; t < lo.y; t++) {
        const int J = (int)g.list[lo.x + t];
        const int j0 = J * TILE;
        const int cnt = min(TILE, g.n - j0);
        __syncwarp();
        if (lane < cnt) P::stage(sj[w][lane], j0 + lane, prm);
        __syncwarp();
        for (int jj = 0; jj < cnt; jj++) P::pair(st, sj[w][jj], j0 + jj, i, valid, prm);
    }
    if (valid) P::finish(st, i, prm);
    if (g.pairs) {
        unsigned c = valid ? (unsigned)P::count(st) : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c) atomicAdd(g.pairs, (unsigned long long)c);
    }
}

template <class P, int WARPS>
int launch_pass(crk_ctx *ctx, int prof_id, bool union_list, const typename P::Params &prm,
                unsigned long long *pairs, cudaStream_t s, const char *what) {
    if (ctx->n == 0) return CRK_OK;
    PassGeom g;
    g.n = ctx->n;
    g.ntiles = ctx->ntiles;
    g.ofs = union_list ? ctx->uofs : ctx->gofs;
    g.list = union_list ? ctx->ulist : ctx->glist;
    g.pairs = pairs;
    prof_begin(ctx, prof_id, s);
    k_pass<P, WARPS><<<grid_for(ctx->ntiles, WARPS), WARPS * 32, 0, s>>>(g, prm);
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, what);
    return CRK_OK;
}

// Pair-sum accumulator: plain FP32, or Kahan-compensated (precision mode 1),
// whose error stays near one rounding of the final sum however much the terms
// cancel (the odd moments and grad m1 = delta m0 + sum V x grad W do).
template <bool COMP>
struct Acc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        if (COMP) {
            float y = v - c;
            float t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += v;
        }
    }
    __device__ __forceinline__ float value() const { return COMP ? s - c : s; }
};

// ---------------------------------------------------------------- list passes



// Warp per tile, lane = particle i; lane i walks its own neighbour list (entry
// k at base + 32 k + lane).  Gather passes walk the first cnt_g[i] entries,
// pair-set passes all cnt_u[i].  P must provide Params, IState, Rec, GATHER,
// PREFETCH, UNROLL, PERSISTENT, ENTRIES (false: the pass reads only its stored entries,
// and `entry` is passed as 0),
//   init(IState&, int i, bool valid, const Params&)
//   load(uint32_t entry, size_t pos, const Params&) -> Rec   (the neighbour's data)
//   pair(IState&, const Rec&, uint32_t entry, size_t pos, bool in_i, const Params&)
//   finish(IState&, int i, const Params&)            (valid lanes only)
struct ListGeom {
    int n, ntiles, kcap;
    const uint32_t *fbase;             // per-tile stored-force base, units of 32 entries
    const uint32_t *len_g, *len_u;
    const int32_t *cnt_g, *cnt_u;
    const uint32_t *ent;
};

// Entry k of a particle's list (gather neighbours k < cnt_g from the front
// columns, the rest from the back columns) and its stored-force position.
// The entries stream once from HBM, the longest latency of the loop, so they
// are always read ahead.  Passes with 16-32-byte records (mostly L1 hits)
// take P::UNROLL entries per iteration: that many independent gathers and
// pair evaluations per lane, the next P::UNROLL entries in flight (measured
// best: 4 for P1 and P2, 3 for P3 and P5).  P4, whose 160-byte record
// already fills the registers, evaluates one pair at a time and instead
// prefetches the record of entry k + 1 and the entry k + 2 (P::PREFETCH),
// alternating two register sets for the record in flight (measured 7%
// faster than copying the prefetched record into the current one).
// passes that declare SKIPPABLE take a device flag (Params::skip, may be null)
template <class P, class = void>
struct has_skip : std::false_type {};
template <class P>
struct has_skip<P, std::void_t<decltype(P::SKIPPABLE)>> : std::bool_constant<P::SKIPPABLE> {};

// passes that declare NOTUNE run their own loop form only (no autotuner variants)
template <class P, class = void>
struct has_notune : std::false_type {};
template <class P>
struct has_notune<P, std::void_t<decltype(P::NOTUNE)>> : std::bool_constant<P::NOTUNE> {};

template <class P>
__device__ __forceinline__ bool pass_skipped(const typename P::Params &prm) {
    if constexpr (has_skip<P>::value) return prm.skip && *(volatile const unsigned long long *)prm.skip;
    return false;
}

// What a lane reads ahead for entry k: its list entry (P::ENTRIES), or, for a
// pass that reads only what an earlier pass stored per entry, that stored
// record (P::Stored, from P::stored(pos)), which then streams from HBM.
template <class P, bool = P::ENTRIES>
struct EntOf {
    using type = uint32_t;
};
template <class P>
struct EntOf<P, false> {
    using type = typename P::Stored;
};

// Entries [k0, mk) of this lane, U per iteration, the warp looping over
// [k0, k1): U independent gathers and pair evaluations in flight per lane and
// the next U entries (or stored records) read ahead.
template <class P, int U, class EntryFn>
__device__ __forceinline__ void list_loop(typename P::IState &st, const typename P::Params &prm, EntryFn entry,
                                          size_t fb, int mg, int k0, int k1, int mk) {
    using Ent = typename EntOf<P>::type;
    auto fetch = [&](int k) -> Ent {
        if constexpr (P::ENTRIES)
            return entry(k);
        else
            return P::stored(fb + (size_t)k * 32, prm);
    };
    Ent en[U] = {};
#pragma unroll
    for (int u = 0; u < U; u++)
        if (k0 + u < mk) en[u] = fetch(k0 + u);
    for (int k = k0; k < k1; k += U) {
        Ent ec[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            ec[u] = en[u];
            if (k + U + u < mk) en[u] = fetch(k + U + u);
        }
        const size_t pos = fb + (size_t)k * 32;
        typename P::Rec r[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            if (k + u < mk) r[u] = P::load(ec[u], pos + 32 * u, prm);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (k + u < mk) P::pair(st, r[u], ec[u], pos + 32 * u, k + u < mg, prm);
    }
}

// list_loop with the neighbour records one iteration ahead as well (RP
// variants): at iteration k the records of iteration k + 1 and the entries
// (or stored records) of iteration k + 2 are in flight while the U pairs of
// iteration k are evaluated, so a record that misses L1 is waited for only if
// it takes longer than a whole iteration.  Same entries, same order: bitwise
// the same sums.
template <class P, int U, class EntryFn>
__device__ __forceinline__ void list_loop_rp(typename P::IState &st, const typename P::Params &prm, EntryFn entry,
                                             size_t fb, int mg, int k0, int k1, int mk) {
    using Ent = typename EntOf<P>::type;
    auto fetch = [&](int k) -> Ent {
        if constexpr (P::ENTRIES)
            return entry(k);
        else
            return P::stored(fb + (size_t)k * 32, prm);
    };
    Ent ec[U] = {}, en[U] = {};
    typename P::Rec rc[U] = {}, rn[U] = {};
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (k0 + u < mk) ec[u] = fetch(k0 + u);
        if (k0 + U + u < mk) en[u] = fetch(k0 + U + u);
    }
#pragma unroll
    for (int u = 0; u < U; u++)
        if (k0 + u < mk) rc[u] = P::load(ec[u], fb + (size_t)(k0 + u) * 32, prm);
    for (int k = k0; k < k1; k += U) {
        Ent eu[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (k + U + u < mk) rn[u] = P::load(en[u], fb + (size_t)(k + U + u) * 32, prm);
            eu[u] = ec[u];
            ec[u] = en[u];
            if (k + 2 * U + u < mk) en[u] = fetch(k + 2 * U + u);
        }
        const size_t pos = fb + (size_t)k * 32;
#pragma unroll
        for (int u = 0; u < U; u++)
            if (k + u < mk) P::pair(st, rc[u], eu[u], pos + 32 * u, k + u < mg, prm);
#pragma unroll
        for (int u = 0; u < U; u++) rc[u] = rn[u];
    }
}

template <class P, int U, bool RP = false>
__device__ __forceinline__ void lpass_tile(const ListGeom &g, const typename P::Params &prm, int tile, int lane) {
    if (pass_skipped<P>(prm)) return;   // the sums were formed by an earlier pass
    const int i = tile * TILE + lane;
    const bool valid = i < g.n;
    typename P::IState st;
    P::init(st, i, valid, prm);
    const uint32_t *col0 = g.ent + (size_t)tile * g.kcap * 32 + lane;
    const size_t fb = (size_t)g.fbase[tile] * 32 + lane;
    // counts beyond kcap only occur in a walk that overflowed (the host then
    // grows kcap and walks again, or discards a replayed step): never read
    // past the tile's columns
    const int len = min((int)(P::GATHER ? g.len_g[tile] : g.len_u[tile]), g.kcap);
    const int mg = valid ? min(g.cnt_g[i], g.kcap) : 0;
    const int my = P::GATHER ? mg : (valid ? min(g.cnt_u[i], g.kcap) : 0);
    auto entry = [&](int k) -> uint32_t {
        const int c = k < mg ? k : g.kcap - 1 - (k - mg);
        return __ldg(col0 + (size_t)c * 32);
    };
    if constexpr (!P::PREFETCH) {
        if constexpr (RP)
            list_loop_rp<P, U>(st, prm, entry, fb, mg, 0, len, my);
        else
            list_loop<P, U>(st, prm, entry, fb, mg, 0, len, my);
    } else {
        // two pairs per iteration: the record in flight alternates between
        // two register sets, so no record is copied from one to the other
        uint32_t e1 = my > 0 ? entry(0) : 0u;
        uint32_t e2 = my > 1 ? entry(1) : 0u;
        typename P::Rec ra{}, rb{};
        if (my > 0) ra = P::load(e1, fb, prm);
        for (int k = 0; k < len; k += 2) {
            const size_t pos = fb + (size_t)k * 32;
            if (k < my) {
                const uint32_t e = e1;
                if (k + 1 < my) rb = P::load(e2, pos + 32, prm);
                e1 = e2;
                if (k + 2 < my) e2 = entry(k + 2);
                P::pair(st, ra, e, pos, k < mg, prm);
            }
            if (k + 1 < my) {
                const uint32_t e = e1;
                if (k + 2 < my) ra = P::load(e2, pos + 64, prm);
                e1 = e2;
                if (k + 3 < my) e2 = entry(k + 3);
                P::pair(st, rb, e, pos + 32, k + 1 < mg, prm);
            }
        }
    }
    if (valid) P::finish(st, i, prm);
}

// Grid form: warp w of block b takes tile order[b WARPS + w] (order null:
// tiles in Morton order).
template <class P, int WARPS, int U, bool RP = false>
__global__ void __launch_bounds__(WARPS * 32) k_lpass(ListGeom g, typename P::Params prm, const int32_t *order) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * WARPS + w;
    if (t >= g.ntiles) return;
    lpass_tile<P, U, RP>(g, prm, order ? order[t] : t, lane);
}

// Persistent form (one warp per block, as many blocks as fit at once): SM s
// owns the contiguous tile range [s chunk, (s+1) chunk) and its warps claim
// tiles from it in order with an atomic counter, so the warps resident on one
// SM work on neighbouring tiles, whose neighbour records they share in L1.  A
// warp whose range is exhausted claims tiles from the other ranges.  Every
// claim is one atomicAdd; a range's counter runs past chunk at most once per
// warp, so the loop is bounded.
template <class P, int U, bool RP = false>
__global__ void __launch_bounds__(32) k_lpass_sm(ListGeom g, typename P::Params prm, uint32_t *next, int nrange,
                                                 int chunk) {
    const int lane = threadIdx.x & 31;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int home = (int)(smid % (unsigned)nrange);
    for (int r = 0; r < nrange; r++) {
        const int range = (home + r) % nrange;
        for (;;) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(&next[range], 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= (uint32_t)chunk) break;
            const long long tile = (long long)range * chunk + t;
            if (tile >= g.ntiles) break;
            lpass_tile<P, U, RP>(g, prm, (int)tile, lane);
        }
    }
}

// Split form, for passes over few tiles (time bins: the leaves ending a step
// at a deep level): S warps share one tile, warp w walking the entry range
// [w chunk, (w+1) chunk) of every lane's list, so a tile's pairs take 1/S of
// the time of one warp walking them all.  Warps w > 0 start from empty sums
// (P::zero); warp 0 merges their partial states in warp order (P::merge,
// deterministic) and finishes.  The stored forces of P4 go to the same entry
// positions as in the other forms; the sums differ from them by rounding.
template <class P>
constexpr int split_warps() {
    return (7 * 32 * sizeof(typename P::IState) <= 44 * 1024) ? 8
           : ((3 * 32 * sizeof(typename P::IState) <= 44 * 1024) ? 4 : 2);
}

template <class P, int S, int U>
__global__ void __launch_bounds__(S * 32) k_lpass_split(ListGeom g, typename P::Params prm, const int32_t *order) {
    using IS = typename P::IState;
    __shared__ __align__(16) unsigned char part[(S - 1) * 32 * sizeof(IS)];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = order[blockIdx.x];
    const int i = tile * TILE + lane;
    const bool valid = i < g.n;
    IS st;
    P::init(st, i, valid, prm);
    if (w > 0) P::zero(st);
    const uint32_t *col0 = g.ent + (size_t)tile * g.kcap * 32 + lane;
    const size_t fb = (size_t)g.fbase[tile] * 32 + lane;
    const int len = min((int)(P::GATHER ? g.len_g[tile] : g.len_u[tile]), g.kcap);
    const int mg = valid ? min(g.cnt_g[i], g.kcap) : 0;
    const int my = P::GATHER ? mg : (valid ? min(g.cnt_u[i], g.kcap) : 0);
    const int chunk = ((len + S - 1) / S + U - 1) / U * U;
    const int k0 = w * chunk, k1 = min(len, k0 + chunk);
    const int mk = min(my, k1);   // this warp's entries of this lane: [k0, mk)
    auto entry = [&](int k) -> uint32_t {
        const int c = k < mg ? k : g.kcap - 1 - (k - mg);
        return __ldg(col0 + (size_t)c * 32);
    };
    list_loop<P, U>(st, prm, entry, fb, mg, k0, k1, mk);
    IS *sp = reinterpret_cast<IS *>(part);
    if (w > 0) sp[(w - 1) * 32 + lane] = st;
    __syncthreads();
    if (w == 0) {
#pragma unroll 1
        for (int v = 1; v < S; v++) P::merge(st, sp[(v - 1) * 32 + lane]);
        if (valid) P::finish(st, i, prm);
    }
}

// merge a partial pair sum into another (the compensated sum keeps the
// partial's correction term)
template <bool C>
__device__ __forceinline__ void merge_acc(Acc<C> &d, const Acc<C> &o) {
    d.add(o.s);
    if (C) d.add(-o.c);
}

// ---------------------------------------------------------------- autotuner
//
// Variants of a list pass: the loop form (U pairs per iteration for the small
// records; U is 1 for P4's prefetching loop) and the order tiles are taken in
// (Morton in the grid; contiguous per-SM ranges in the persistent form;
// longest list first in the grid).  Every variant visits each particle's list
// in the same order, so all give bitwise identical results; the tuner times
// each once on the first evaluation after crk_autotune(ctx, 1) and keeps the
// fastest per pass.
enum { ORD_GRID = 0, ORD_SM = 1, ORD_LONGEST = 2 };
struct LVariant {
    int U, ord;
    int warps;   // tiles per CTA in the grid form (32 particles each); 0 = the pass's own
    bool rp;     // records one iteration ahead (list_loop_rp)
    bool tma;    // records brought into shared memory by TMA gathers (passes with P::TMA)
};
// 0-3: grid, U = 1..4; 4-7: longest first, U = 1..4; 8: per-SM ranges;
// 9-12: grid with the pass's own U and CTAs of 1, 2, 4, 8 tiles (32-256 particles);
// 13-16: grid, U = 1..4, records one iteration ahead, CTAs of one tile;
// 17-20: the same with the pass's own CTA width (passes without their own
// record prefetch: all but P4); 21: records by TMA gathers (P4); 22: per-SM
// ranges with the pass's own U and records one iteration ahead (all but P4)
__host__ __device__ constexpr LVariant lvariant(int v) {
    return v < 4 ? LVariant{v + 1, ORD_GRID, 0, false, false}
                 : (v < 8 ? LVariant{v - 3, ORD_LONGEST, 0, false, false}
                          : (v == 8 ? LVariant{1, ORD_SM, 0, false, false}
                                    : (v < 13 ? LVariant{0, ORD_GRID, 1 << (v - 9), false, false}
                                              : (v < 17 ? LVariant{v - 12, ORD_GRID, 1, true, false}
                                                        : (v < 21 ? LVariant{v - 16, ORD_GRID, 0, true, false}
                                                                  : (v == 21 ? LVariant{1, ORD_GRID, 0, false, true}
                                                                             : LVariant{0, ORD_SM, 0, true, false}))))));
}

// passes with a TMA-fed variant (21)
template <class P, class = void>
struct has_tma : std::false_type {};
template <class P>
struct has_tma<P, std::void_t<decltype(P::TMA)>> : std::bool_constant<P::TMA> {};

int tile_order_by_length(crk_ctx *ctx, cudaStream_t s);   // ctx->tile_order, longest pair-set list first

template <class P, int WARPS, int U>
static void launch_variant_u(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, int ord,
                             cudaStream_t s) {
    if (ord == ORD_SM) {
        static int per_sm = 0;
        if (!per_sm) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lpass_sm<P, U>, 32, 0) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
        }
        const int nrange = ctx->nsm > 0 ? (ctx->nsm < 1024 ? ctx->nsm : 1024) : 1;
        const int chunk = (ctx->ntiles + nrange - 1) / nrange;
        cudaMemsetAsync(ctx->sm_next, 0, sizeof(uint32_t) * nrange, s);
        k_lpass_sm<P, U><<<nrange * per_sm, 32, 0, s>>>(g, prm, ctx->sm_next, nrange, chunk);
    } else {
        k_lpass<P, WARPS, U><<<grid_for(ctx->ntiles, WARPS), WARPS * 32, 0, s>>>(
            g, prm, ord == ORD_LONGEST ? ctx->tile_order : nullptr);
    }
}

// per-SM tile ranges, the pass's own entries per iteration, records one
// iteration ahead
template <class P>
static void launch_sm_rp(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, cudaStream_t s) {
    constexpr int U = P::UNROLL;
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lpass_sm<P, U, true>, 32, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    const int nrange = ctx->nsm > 0 ? (ctx->nsm < 1024 ? ctx->nsm : 1024) : 1;
    const int chunk = (ctx->ntiles + nrange - 1) / nrange;
    cudaMemsetAsync(ctx->sm_next, 0, sizeof(uint32_t) * nrange, s);
    k_lpass_sm<P, U, true><<<nrange * per_sm, 32, 0, s>>>(g, prm, ctx->sm_next, nrange, chunk);
}

template <class P, int W>
static void launch_width(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, cudaStream_t s) {
    constexpr int U = P::PREFETCH ? 1 : P::UNROLL;
    k_lpass<P, W, U><<<grid_for(ctx->ntiles, W), W * 32, 0, s>>>(g, prm, nullptr);
}

template <class P, int W, int U>
static void launch_rp(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, cudaStream_t s) {
    k_lpass<P, W, U, true><<<grid_for(ctx->ntiles, W), W * 32, 0, s>>>(g, prm, nullptr);
}

template <class P, int W>
static void launch_rp_u(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, int U, cudaStream_t s) {
    switch (U) {
    case 1: launch_rp<P, W, 1>(ctx, g, prm, s); break;
    case 2: launch_rp<P, W, 2>(ctx, g, prm, s); break;
    case 3: launch_rp<P, W, 3>(ctx, g, prm, s); break;
    default: launch_rp<P, W, 4>(ctx, g, prm, s); break;
    }
}

template <class P, int WARPS>
static int launch_variant(crk_ctx *ctx, const ListGeom &g, const typename P::Params &prm, int v, cudaStream_t s) {
    const LVariant lv = lvariant(v);
    if (lv.tma) {
        if constexpr (has_tma<P>::value) return P::launch_tma(ctx, g, prm, s);
        return CRK_OK;
    }
    if (lv.rp && lv.ord == ORD_SM) {
        if constexpr (!P::PREFETCH) launch_sm_rp<P>(ctx, g, prm, s);
        return CRK_OK;
    }
    if (lv.rp) {   // records one iteration ahead (passes without their own prefetch)
        if constexpr (!P::PREFETCH) {
            if (lv.warps == 1)
                launch_rp_u<P, 1>(ctx, g, prm, lv.U, s);
            else
                launch_rp_u<P, WARPS>(ctx, g, prm, lv.U, s);
        }
        return CRK_OK;
    }
    if (lv.warps) {   // CTA width variants (the pass's own loop form)
        switch (lv.warps) {
        case 1: launch_width<P, 1>(ctx, g, prm, s); break;
        case 2: launch_width<P, 2>(ctx, g, prm, s); break;
        case 4: launch_width<P, 4>(ctx, g, prm, s); break;
        default: launch_width<P, 8>(ctx, g, prm, s); break;
        }
        return CRK_OK;
    }
    if (lv.ord == ORD_LONGEST) {
        int rc = tile_order_by_length(ctx, s);
        if (rc) return rc;
    }
    if constexpr (P::PREFETCH) {
        launch_variant_u<P, WARPS, 1>(ctx, g, prm, lv.ord, s);
    } else {
        switch (lv.U) {
        case 1: launch_variant_u<P, WARPS, 1>(ctx, g, prm, lv.ord, s); break;
        case 2: launch_variant_u<P, WARPS, 2>(ctx, g, prm, lv.ord, s); break;
        case 3: launch_variant_u<P, WARPS, 3>(ctx, g, prm, lv.ord, s); break;
        default: launch_variant_u<P, WARPS, 4>(ctx, g, prm, lv.ord, s); break;
        }
    }
    return CRK_OK;
}

// the measured default of each pass (before or without tuning)
template <class P>
constexpr int default_variant() {
    return P::PREFETCH ? (P::PERSISTENT ? 8 : 0) : P::UNROLL - 1;
}

template <class P>
constexpr bool variant_applies(int v) {
    if (lvariant(v).tma) return has_tma<P>::value;
    if (lvariant(v).rp) return !P::PREFETCH;
    return P::PREFETCH ? (lvariant(v).U <= 1) : true;
}

// tune_slot: the autotuner's record for this pass (default: its profiling id;
// a pass with a different record layout, such as the two-kick P5, keeps its own)
template <class P, int WARPS, int MINB = 1>
int launch_lpass(crk_ctx *ctx, int prof_id, const typename P::Params &prm, cudaStream_t s, const char *what,
                 int tune_slot = -1) {
    const int ts = tune_slot >= 0 ? tune_slot : prof_id;
    if (ctx->n == 0) return CRK_OK;
    if (!ctx->lists_valid) return crk_set_error(ctx, CRK_ESTATE, "%s: neighbour lists are not built", what);
    ListGeom g{ctx->n, ctx->ntiles, ctx->kcap, ctx->tbase, ctx->len_g, ctx->len_u, ctx->cnt_g, ctx->cnt_u,
               ctx->ent};
    int rc;
    if (ctx->act) {
        // the tiles ctx->act[0 .. nact) only (time bins): grid form over that
        // list, each pass's default loop form, no tuning
        if (ctx->nact == 0) return CRK_OK;
        g.ntiles = ctx->nact;
        constexpr int U = P::PREFETCH ? 1 : P::UNROLL;
        prof_begin(ctx, prof_id, s);
        const int nsm = ctx->nsm > 0 ? ctx->nsm : 152;
        constexpr int S = split_warps<P>();
        if (ctx->nact < 8 * nsm)   // few tiles: S warps per tile
            k_lpass_split<P, S, U><<<ctx->nact, S * 32, 0, s>>>(g, prm, ctx->act);
        else
            k_lpass<P, WARPS, U><<<grid_for(ctx->nact, WARPS), WARPS * 32, 0, s>>>(g, prm, ctx->act);
        ++ctx->launches;
        prof_end(ctx, s);
        CRK_LAUNCH_CHECK(ctx, what);
        return CRK_OK;
    }
    if constexpr (has_notune<P>::value) {
        constexpr int U = P::PREFETCH ? 1 : P::UNROLL;
        prof_begin(ctx, prof_id, s);
        k_lpass<P, WARPS, U><<<grid_for(ctx->ntiles, WARPS), WARPS * 32, 0, s>>>(g, prm, nullptr);
        ++ctx->launches;
        prof_end(ctx, s);
        CRK_LAUNCH_CHECK(ctx, what);
        return CRK_OK;
    }
    if (ctx->tune_on && !ctx->tune_done[ts]) {
        // time every applicable variant once (each recomputes the same outputs)
        float best = 3.0e38f;
        int bestv = default_variant<P>();
        for (int v = 0; v < NVAR; v++) {
            // the TMA-fed variant is measured 6x slower than the L1 forms on
            // GB300: it runs only when pinned (crk_tune_set)
            if (!variant_applies<P>(v) || lvariant(v).tma) continue;
            CRK_CUDA(ctx, cudaEventRecord(ctx->tune_ev[0], s));
            rc = launch_variant<P, WARPS>(ctx, g, prm, v, s);
            if (rc) return rc;
            CRK_CUDA(ctx, cudaEventRecord(ctx->tune_ev[1], s));
            ++ctx->launches;
            CRK_LAUNCH_CHECK(ctx, what);
            CRK_CUDA(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
            float ms = 0.f;
            CRK_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->tune_ev[0], ctx->tune_ev[1]));
            if (ms < best) {
                best = ms;
                bestv = v;
            }
        }
        ctx->tune_choice[ts] = bestv;
        ctx->tune_ms[ts] = best;
        ctx->tune_done[ts] = 1;
    }
    const int v = ctx->tune_choice[ts] >= 0 ? ctx->tune_choice[ts] : default_variant<P>();
    if (!variant_applies<P>(v))   // only a variant pinned by crk_tune_set can be one the pass lacks
        return crk_set_error(ctx, CRK_EINVAL, "%s: the pass has no variant %d", what, v);
    prof_begin(ctx, prof_id, s);
    rc = launch_variant<P, WARPS>(ctx, g, prm, v, s);
    if (rc) return rc;
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, what);
    return CRK_OK;
}

// ---------------------------------------------------------------- kernel maths

// C4 Wendland kernel (eq:C4) with eta = r/h and t = 1 - eta:
//   W = 495/(32 pi h^3) t^6 (1 + 6 eta + 35/3 eta^2)
//   grad_i W = -1155/(4 pi h^5) (1 + 5 eta) t^5 x_ij
// The constants are evaluated from their definitions at compile time (a
// hand-typed 1155/(4 pi) was once 6e-7 off, which the cancellation in the
// diagonal of grad m1 = delta m0 + cG sum V x x Gu amplified ~100-fold).
constexpr double KW_D = 495.0 / (32.0 * PI_D);
constexpr double KG_D = 1155.0 / (4.0 * PI_D);
constexpr float KW = (float)KW_D;         // 495 / (32 pi)
constexpr float KG = (float)KG_D;         // 1155 / (4 pi)
constexpr float K35_3 = (float)(35.0 / 3.0);
constexpr float K4PI_3 = (float)(4.0 * PI_D / 3.0);   // eq:hi

// Two float4 of a record in one 256-bit read-only load (p on a 32-byte
// boundary): one L1 sector per lane per instruction.
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

struct Sep {
    float x, y, z, r2, r;
};

__device__ __forceinline__ Sep separation(int dx, int dy, int dz) {
    Sep s;
    s.x = (float)dx * TWO_M32;
    s.y = (float)dy * TWO_M32;
    s.z = (float)dz * TWO_M32;
    s.r2 = fmaf(s.x, s.x, fmaf(s.y, s.y, s.z * s.z));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s.r) : "f"(s.r2));
    return s;
}

}  // namespace crk
