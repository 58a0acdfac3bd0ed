// crk_cells.cu -- chaining-mesh binning and interaction lists (CRK-HACC Sec. 2.3:
// particles binned into chaining-mesh cells, flattened contiguous leaves with
// bounding boxes grown by the maximal smoothing length, and interaction lists
// assembled once per hydro step and reused by every hydro kernel).
//
// GB300 layout: 30-bit Morton keys of the fixed-point coordinates, a stable LSD
// radix sort (8-bit digits, per-warp stable ranking with match_any), sorted
// SoA particle records, tiles of 32 consecutive sorted particles (one warp),
// an implicit binary tree over the Morton-ordered tiles, and per-tile lists of
// neighbour tiles found by a depth-first walk of that tree with exact
// fixed-point gap tests (never drops a pair of the neighbour predicate).
#include "crk_internal.cuh"

#include <string.h>
#include <math.h>

namespace crk {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ keys

// Per particle t of the input order: fixed-point record, Morton key, max h.
// Invalid records (coordinates outside [0,1) or non-finite, h outside
// (0, 1/3)) are counted and replaced by a harmless record.
__global__ void k_keys(int n, const float4 *__restrict__ pos, uint32_t *__restrict__ key,
                       int32_t *__restrict__ idx, uint4 *__restrict__ q_tmp,
                       float *__restrict__ h_tmp, unsigned long long *counters, int hilbert) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t hbits = 0u;
    if (t < n) {
        float4 p = pos[t];
        bool ok = (p.x >= 0.f && p.x < 1.f) && (p.y >= 0.f && p.y < 1.f) && (p.z >= 0.f && p.z < 1.f) &&
                  ((double)p.w > 0.0 && (double)p.w < 1.0 / 3.0);
        if (!ok) {
            atomicAdd(&counters[CNT_ERR_INPUT], 1ull);
            p = make_float4(0.f, 0.f, 0.f, 0.01f);
        }
        uint4 q = make_uint4(to_fixed(p.x), to_fixed(p.y), to_fixed(p.z), to_fixed(p.w));
        q_tmp[t] = q;
        h_tmp[t] = p.w;
        key[t] = hilbert ? hilbert30(q.x, q.y, q.z) : morton30(q.x, q.y, q.z);
        idx[t] = t;
        hbits = __float_as_uint(p.w);   // h > 0: the bits order like the values
    }
    // max h: one atomic per warp, not one per particle on a single address
    hbits = __reduce_max_sync(0xffffffffu, hbits);
    if ((threadIdx.x & 31) == 0 && hbits) atomicMax(&counters[CNT_HMAX], (unsigned long long)hbits);
}

// ------------------------------------------------------------------ radix sort

constexpr int RS_WARPS = 8;
constexpr int RS_PER_WARP = 512;
constexpr int RS_ITEMS = RS_WARPS * RS_PER_WARP;   // keys per block

__global__ void __launch_bounds__(256) k_rs_hist(int n, const uint32_t *__restrict__ key, int shift,
                                                 uint32_t *__restrict__ hist, int nblocks) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_ITEMS;
    for (int k = threadIdx.x; k < RS_ITEMS; k += 256) {
        int i = base + k;
        if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: warp w of block b owns the contiguous items
// [b*RS_ITEMS + w*RS_PER_WARP, +RS_PER_WARP); within a warp, items are ranked in
// index order with match_any, so equal digits keep their input order.
__global__ void __launch_bounds__(256) k_rs_scatter(int n, const uint32_t *__restrict__ key_in,
                                                    const int32_t *__restrict__ val_in,
                                                    uint32_t *__restrict__ key_out,
                                                    int32_t *__restrict__ val_out, int shift,
                                                    const uint32_t *__restrict__ hist_scan,
                                                    int nblocks) {
    __shared__ uint32_t off[RS_WARPS][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) off[w][d] = 0;
    __syncwarp();
    int wbase = blockIdx.x * RS_ITEMS + w * RS_PER_WARP;
    for (int k = 0; k < RS_PER_WARP / 32; k++) {
        int i = wbase + k * 32 + lane;
        bool v = i < n;
        uint32_t d = v ? ((key_in[i] >> shift) & 255u) : 256u + lane;
        unsigned peers = __match_any_sync(FULL, d);
        if (v && lane == __ffs(peers) - 1) off[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;
        uint32_t run = hist_scan[d * nblocks + blockIdx.x];
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t c = off[ww][d];
            off[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    unsigned lt = lanemask_lt();
    for (int k = 0; k < RS_PER_WARP / 32; k++) {
        int i = wbase + k * 32 + lane;
        bool v = i < n;
        uint32_t kk = v ? key_in[i] : 0u;
        uint32_t d = v ? ((kk >> shift) & 255u) : 256u + lane;
        unsigned peers = __match_any_sync(FULL, d);
        uint32_t base = v ? off[w][d] : 0u;
        __syncwarp();
        if (v) {
            uint32_t pos = base + __popc(peers & lt);
            key_out[pos] = kk;
            val_out[pos] = val_in[i];
            if (lane == __ffs(peers) - 1) off[w][d] = base + __popc(peers);
        }
        __syncwarp();
    }
}

// Exclusive scan, 4096 items per block.
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t *__restrict__ in,
                                                     uint32_t *__restrict__ out, int count,
                                                     uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t wt[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = blockIdx.x * 4096 + threadIdx.x * 4;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        int i = base + k;
        v[k] = i < count ? in[i] : 0u;
        s += v[k];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        wt[lane] = t;
    }
    __syncthreads();
    uint32_t excl = x - s + (warp > 0 ? wt[warp - 1] : 0u);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        int i = base + k;
        if (i < count) out[i] = excl;
        excl += v[k];
    }
    if (threadIdx.x == 1023 && block_sums) block_sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(uint32_t *__restrict__ out, int count, const uint32_t *__restrict__ offs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] += offs[i / 4096];
}

// exclusive scan of count <= 4096*4096 values (ctx->scan_tmp holds >= 2*4096 words)
int scan_u32(crk_ctx *ctx, const uint32_t *in, uint32_t *out, int count, cudaStream_t s) {
    uint32_t *scratch = ctx->scan_tmp;
    int nb = grid_for(count, 4096);
    if (nb > 4096) return crk_set_error(ctx, CRK_ECAPACITY, "scan of %d items exceeds 2 levels", count);
    k_scan_block<<<nb, 1024, 0, s>>>(in, out, count, scratch);
    ++ctx->launches;
    if (nb > 1) {
        k_scan_block<<<1, 1024, 0, s>>>(scratch, scratch + 4096, nb, nullptr);
        ++ctx->launches;
        k_scan_add<<<grid_for(count, 256), 256, 0, s>>>(out, count, scratch + 4096);
        ++ctx->launches;
    }
    CRK_LAUNCH_CHECK(ctx, "scan");
    return CRK_OK;
}

// Stable sort of (key_a, idx_a) by the low `bits` bits of key; result in key_a/idx_a.
static int radix_sort(crk_ctx *ctx, int n, int bits, cudaStream_t s) {
    int nblocks = grid_for(n, RS_ITEMS);
    int passes = (bits + 7) / 8;
    if (passes & 1) passes++;   // even number of passes leaves the result in the _a buffers
    uint32_t *kin = ctx->key_a, *kout = ctx->key_b;
    int32_t *vin = ctx->idx_a, *vout = ctx->idx_b;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_rs_hist<<<nblocks, 256, 0, s>>>(n, kin, shift, ctx->hist, nblocks);
        ++ctx->launches;
        int rc = scan_u32(ctx, ctx->hist, ctx->hist, 256 * nblocks, s);
        if (rc) return rc;
        k_rs_scatter<<<nblocks, 256, 0, s>>>(n, kin, vin, kout, vout, shift, ctx->hist, nblocks);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "radix sort");
        uint32_t *tk = kin; kin = kout; kout = tk;
        int32_t *tv = vin; vin = vout; vout = tv;
    }
    return CRK_OK;
}

// ------------------------------------------------------------------ recursive coordinate bisection
//
// tile_order 2: the Morton order is refined by recursive coordinate bisection
// into leaves of at most `leaf` particles (crk_params.rcb_leaf: 32 = one tile,
// or the paper's 128 / 256, whose tiles are then cut from the order the
// splits leave inside each leaf).  A segment [a, b) of more than `leaf` particles splits
// at nl = 32 ceil(ceil((b - a)/2) / 32) (every left part a whole number of
// tiles) along the longest axis of its fixed-point box: its particles are
// binned into 256 equal slices of that box, the slice holding the nl-th
// particle is the median slice, and a stable partition puts the slices
// below it first, then the median slice, then the slices above, so the
// first nl particles are the lower part.  Level by level, all segments at
// once; within a leaf the Morton order stays.

constexpr int RCB_BINS = 256;

__host__ __device__ __forceinline__ int rcb_left(int size) { return ((size + 1) / 2 + 31) / 32 * 32; }

// the segment of slot s after `level` splits: start a, size, index (path bits)
__device__ __forceinline__ bool rcb_segment(int n, int level, int leaf, int s, int &a, int &size, int &path) {
    a = 0;
    size = n;
    path = 0;
    for (int l = 0; l < level; l++) {
        if (size <= leaf) return false;
        const int nl = rcb_left(size);
        if (s < a + nl) {
            size = nl;
            path = 2 * path;
        } else {
            a += nl;
            size -= nl;
            path = 2 * path + 1;
        }
    }
    return size > leaf;
}

// per slot: its segment (start, index; -1 when the segment does not split)
// and the segment's box (one atomic per segment a warp touches)
__global__ void k_rcb_box(int n, int level, int leaf, const int32_t *__restrict__ perm, const uint4 *__restrict__ q,
                          int32_t *__restrict__ seg_a, int32_t *__restrict__ seg_id, uint32_t *__restrict__ blo,
                          uint32_t *__restrict__ bhi, int32_t *__restrict__ bsize) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int a = 0, size = 0, path = -1;
    bool act = false;
    uint4 p = make_uint4(0, 0, 0, 0);
    if (s < n) {
        act = rcb_segment(n, level, leaf, s, a, size, path);
        if (!act) path = -1;
        seg_a[s] = a;
        seg_id[s] = path;
        p = q[perm[s]];
    }
    const unsigned peers = __match_any_sync(FULL, path);
    uint32_t lx = p.x, ly = p.y, lz = p.z, hx = p.x, hy = p.y, hz = p.z;
    for (int k = 0; k < 32; k++) {
        const uint32_t ox = __shfl_sync(FULL, p.x, k), oy = __shfl_sync(FULL, p.y, k), oz = __shfl_sync(FULL, p.z, k);
        if ((peers >> k) & 1u) {
            lx = min(lx, ox); ly = min(ly, oy); lz = min(lz, oz);
            hx = max(hx, ox); hy = max(hy, oy); hz = max(hz, oz);
        }
    }
    if (act && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
        atomicMin(blo + 3 * path, lx); atomicMin(blo + 3 * path + 1, ly); atomicMin(blo + 3 * path + 2, lz);
        atomicMax(bhi + 3 * path, hx); atomicMax(bhi + 3 * path + 1, hy); atomicMax(bhi + 3 * path + 2, hz);
        bsize[path] = size;
    }
}

__device__ __forceinline__ int rcb_axis(const uint32_t *lo, const uint32_t *hi, int path, uint32_t &l0,
                                        unsigned long long &ext) {
    const uint32_t e0 = hi[3 * path] - lo[3 * path], e1 = hi[3 * path + 1] - lo[3 * path + 1],
                   e2 = hi[3 * path + 2] - lo[3 * path + 2];
    int ax = 0;
    uint32_t m = e0;
    if (e1 > m) { ax = 1; m = e1; }
    if (e2 > m) { ax = 2; m = e2; }
    l0 = lo[3 * path + ax];
    ext = (unsigned long long)m + 1ull;
    return ax;
}

// slice of every particle along its segment's axis, and the slice counts
__global__ void k_rcb_hist(int n, const int32_t *__restrict__ perm, const uint4 *__restrict__ q,
                           const int32_t *__restrict__ seg_id, const uint32_t *__restrict__ blo,
                           const uint32_t *__restrict__ bhi, uint32_t *__restrict__ bin, uint32_t *__restrict__ hist) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int path = seg_id[s];
    if (path < 0) return;
    uint32_t l0;
    unsigned long long ext;
    const int ax = rcb_axis(blo, bhi, path, l0, ext);
    const uint4 p = q[perm[s]];
    const uint32_t c = ax == 0 ? p.x : (ax == 1 ? p.y : p.z);
    const uint32_t b = (uint32_t)(((unsigned long long)(c - l0) * RCB_BINS) / ext);
    bin[s] = b;
    atomicAdd(hist + (size_t)path * RCB_BINS + b, 1u);
}

// per segment (warp): the median slice and the counts below it and in it
__global__ void k_rcb_pick(int nseg, const int32_t *__restrict__ bsize, const uint32_t *__restrict__ hist,
                           uint32_t *__restrict__ pick) {
    const int lane = threadIdx.x & 31;
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nseg) return;
    const int size = bsize[g];
    if (size <= TILE) return;
    const uint32_t nl = (uint32_t)rcb_left(size);
    uint32_t v[RCB_BINS / 32], sum = 0;
#pragma unroll
    for (int k = 0; k < RCB_BINS / 32; k++) {
        v[k] = hist[(size_t)g * RCB_BINS + lane * (RCB_BINS / 32) + k];
        sum += v[k];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    uint32_t below = x - sum;   // particles in the slices before this lane's
    int found = -1;
    uint32_t c0 = 0, c1 = 0;
#pragma unroll
    for (int k = 0; k < RCB_BINS / 32; k++) {
        if (found < 0 && below + v[k] >= nl) {
            found = lane * (RCB_BINS / 32) + k;
            c0 = below;
            c1 = v[k];
        }
        below += v[k];
    }
    const unsigned m = __ballot_sync(FULL, found >= 0);
    if (lane == __ffs(m) - 1) {
        pick[3 * g] = (uint32_t)found;
        pick[3 * g + 1] = c0;
        pick[3 * g + 2] = c1;
    }
}

__global__ void k_rcb_flags(int n, const int32_t *__restrict__ seg_id, const uint32_t *__restrict__ bin,
                            const uint32_t *__restrict__ pick, uint32_t *__restrict__ f0, uint32_t *__restrict__ f1) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int path = seg_id[s];
    uint32_t a = 0, b = 0;
    if (path >= 0) {
        const uint32_t m = pick[3 * path], v = bin[s];
        a = v < m;
        b = v == m;
    }
    f0[s] = a;
    f1[s] = b;
}

// stable three-way partition of every splitting segment (below, median, above)
__global__ void k_rcb_scatter(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ seg_a,
                              const int32_t *__restrict__ seg_id, const uint32_t *__restrict__ bin,
                              const uint32_t *__restrict__ pick, const uint32_t *__restrict__ r0,
                              const uint32_t *__restrict__ r1, int32_t *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int path = seg_id[s];
    int d = s;
    if (path >= 0) {
        const int a = seg_a[s];
        const uint32_t m = pick[3 * path], v = bin[s];
        const int k0 = (int)(r0[s] - r0[a]), k1 = (int)(r1[s] - r1[a]);
        const int c0 = (int)pick[3 * path + 1], c1 = (int)pick[3 * path + 2];
        d = v < m ? a + k0 : (v == m ? a + c0 + k1 : a + c0 + c1 + (s - a - k0 - k1));
    }
    out[d] = perm[s];
}

template <class T>
static int rcb_grow(crk_ctx *ctx, T **p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    CRK_CUDA(ctx, cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)));
    ++ctx->alloc_gen;
    return CRK_OK;
}

static int ensure_rcb(crk_ctx *ctx, int n, int nseg) {
    int rc = CRK_OK;
    if (n > ctx->cap_rcb || nseg > ctx->cap_rcb_seg) {
        ctx->cap_rcb = 0;
        ctx->cap_rcb_seg = 0;
        rc = rcb_grow(ctx, &ctx->rcb_a, n);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_id, n);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_bin, n);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_f, 4 * (size_t)n);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_lo, 3 * (size_t)nseg);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_hi, 3 * (size_t)nseg);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_size, nseg);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_pick, 3 * (size_t)nseg);
        if (!rc) rc = rcb_grow(ctx, &ctx->rcb_hist, (size_t)RCB_BINS * nseg);
        if (rc) return rc;
        ctx->cap_rcb = n;
        ctx->cap_rcb_seg = nseg;
    }
    return CRK_OK;
}

void rcb_free(crk_ctx *ctx) {
    void *ps[] = {ctx->rcb_a, ctx->rcb_id, ctx->rcb_size, ctx->rcb_bin, ctx->rcb_f, ctx->rcb_lo, ctx->rcb_hi,
                  ctx->rcb_pick, ctx->rcb_hist};
    for (void *p : ps)
        if (p) cudaFree(p);
    ctx->rcb_a = ctx->rcb_id = ctx->rcb_size = nullptr;
    ctx->rcb_bin = ctx->rcb_f = ctx->rcb_lo = ctx->rcb_hi = ctx->rcb_pick = ctx->rcb_hist = nullptr;
    ctx->cap_rcb = ctx->cap_rcb_seg = 0;
}

__global__ void k_fill_u32(long long count, uint32_t v, uint32_t *out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) out[k] = v;
}

// Refine the sorted order idx_a (input indices) by recursive coordinate
// bisection of the fixed-point records q_tmp (input order).
static int rcb_refine(crk_ctx *ctx, int n, cudaStream_t s) {
    const int leaf = ctx->p.rcb_leaf;
    int levels = 0;
    for (int size = n; size > leaf; size = rcb_left(size)) levels++;   // the largest segment goes left
    int rc = ensure_rcb(ctx, n, 1 << (levels > 0 ? levels - 1 : 0));
    if (rc) return rc;
    int32_t *cur = ctx->idx_a, *nxt = ctx->idx_b;
    uint32_t *f0 = ctx->rcb_f, *f1 = ctx->rcb_f + n, *r0 = ctx->rcb_f + 2 * (size_t)n, *r1 = ctx->rcb_f + 3 * (size_t)n;
    const int g = grid_for(n, 256);
    for (int L = 0; L < levels; L++) {
        const int nseg = 1 << L;
        k_fill_u32<<<grid_for(3ll * nseg, 256), 256, 0, s>>>(3ll * nseg, 0xffffffffu, ctx->rcb_lo);
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->rcb_hi, 0, sizeof(uint32_t) * 3 * (size_t)nseg, s));
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->rcb_size, 0, sizeof(int32_t) * (size_t)nseg, s));
        CRK_CUDA(ctx, cudaMemsetAsync(ctx->rcb_hist, 0, sizeof(uint32_t) * RCB_BINS * (size_t)nseg, s));
        k_rcb_box<<<g, 256, 0, s>>>(n, L, leaf, cur, ctx->q_tmp, ctx->rcb_a, ctx->rcb_id, ctx->rcb_lo, ctx->rcb_hi,
                                    ctx->rcb_size);
        k_rcb_hist<<<g, 256, 0, s>>>(n, cur, ctx->q_tmp, ctx->rcb_id, ctx->rcb_lo, ctx->rcb_hi, ctx->rcb_bin,
                                     ctx->rcb_hist);
        k_rcb_pick<<<grid_for(32ll * nseg, 256), 256, 0, s>>>(nseg, ctx->rcb_size, ctx->rcb_hist, ctx->rcb_pick);
        k_rcb_flags<<<g, 256, 0, s>>>(n, ctx->rcb_id, ctx->rcb_bin, ctx->rcb_pick, f0, f1);
        ctx->launches += 5;
        CRK_LAUNCH_CHECK(ctx, "bisection");
        rc = scan_u32(ctx, f0, r0, n, s);
        if (!rc) rc = scan_u32(ctx, f1, r1, n, s);
        if (rc) return rc;
        k_rcb_scatter<<<g, 256, 0, s>>>(n, cur, ctx->rcb_a, ctx->rcb_id, ctx->rcb_bin, ctx->rcb_pick, r0, r1, nxt);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "bisection");
        int32_t *t = cur; cur = nxt; nxt = t;
    }
    if (cur != ctx->idx_a)
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->idx_a, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    return CRK_OK;
}

// ------------------------------------------------------------------ sorted records

__global__ void k_gather_sorted(int n, const int32_t *__restrict__ idx, const uint4 *__restrict__ q_tmp,
                                const float *__restrict__ h_tmp, const int32_t *__restrict__ base_perm,
                                uint4 *__restrict__ q4, float *__restrict__ hs,
                                int32_t *__restrict__ perm_out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = idx[s];
    q4[s] = q_tmp[i];
    hs[s] = h_tmp[i];
    perm_out[s] = base_perm ? base_perm[i] : i;
}

// ------------------------------------------------------------------ tiles and tree

// Tile boxes as periodic arcs: per axis the smallest arc around the tile's
// first particle that holds every particle, lo = q_0 + min_k d_k and
// hi = q_0 + max_k d_k (mod 2^32) with d_k = (int)(q_k - q_0).  For a tile of
// the Morton order this is its min/max box; a tile whose particles drifted
// across the periodic boundary (time bins keep tiles between sorts) gets an
// arc with lo > hi instead of a box spanning the whole period.
__global__ void k_tiles(int n, int ntiles, const uint4 *__restrict__ q4, uint4 *__restrict__ lo,
                        uint4 *__restrict__ hi, const int32_t *__restrict__ sbox, uint32_t *__restrict__ nbox) {
    int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (tile >= ntiles) return;
    int s = tile * TILE + lane;
    bool v = s < n;
    uint4 q = v ? q4[s] : make_uint4(0, 0, 0, 0);
    const uint32_t rx = __shfl_sync(FULL, q.x, 0), ry = __shfl_sync(FULL, q.y, 0), rz = __shfl_sync(FULL, q.z, 0);
    const int dx = v ? (int)(q.x - rx) : 0, dy = v ? (int)(q.y - ry) : 0, dz = v ? (int)(q.z - rz) : 0;
    uint32_t xl = rx + (uint32_t)__reduce_min_sync(FULL, dx);
    uint32_t yl = ry + (uint32_t)__reduce_min_sync(FULL, dy);
    uint32_t zl = rz + (uint32_t)__reduce_min_sync(FULL, dz);
    uint32_t xh = rx + (uint32_t)__reduce_max_sync(FULL, dx);
    uint32_t yh = ry + (uint32_t)__reduce_max_sync(FULL, dy);
    uint32_t zh = rz + (uint32_t)__reduce_max_sync(FULL, dz);
    uint32_t Hm = __reduce_max_sync(FULL, v ? q.w : 0u);
    uint32_t c = __popc(__ballot_sync(FULL, v));
    if (lane == 0) {
        lo[tile] = make_uint4(xl, yl, zl, Hm);
        hi[tile] = make_uint4(xh, yh, zh, c);
    }
    if (sbox) {   // batched boxes: the range of boxes the tile's particles belong to
        uint32_t b = v ? (uint32_t)sbox[s] : 0u;
        uint32_t bl = __reduce_min_sync(FULL, v ? b : 0xffffu);
        uint32_t bh = __reduce_max_sync(FULL, v ? b : 0u);
        if (lane == 0) nbox[tile] = bl | (bh << 16);
    }
}

__device__ __forceinline__ bool box_ranges_meet(uint32_t a, uint32_t b) {
    return (a & 0xffffu) <= (b >> 16) && (b & 0xffffu) <= (a >> 16);
}

// Inner tree nodes hold plain intervals: a child arc that wraps (lo > hi) is
// widened to the whole axis, which keeps every node a superset of its tiles.
__device__ __forceinline__ void unwrap_arcs(uint4 &l, uint4 &h) {
    if (l.x > h.x) { l.x = 0u; h.x = 0xffffffffu; }
    if (l.y > h.y) { l.y = 0u; h.y = 0xffffffffu; }
    if (l.z > h.z) { l.z = 0u; h.z = 0xffffffffu; }
}

__global__ void k_tree_level(const uint4 *__restrict__ clo, const uint4 *__restrict__ chi, int ccnt,
                             uint4 *__restrict__ plo, uint4 *__restrict__ phi, int pcnt,
                             const uint32_t *__restrict__ cbox, uint32_t *__restrict__ pbox) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= pcnt) return;
    uint4 l = clo[2 * k], h = chi[2 * k];
    uint32_t b = cbox ? cbox[2 * k] : 0u;
    unwrap_arcs(l, h);
    if (2 * k + 1 < ccnt) {
        uint4 l2 = clo[2 * k + 1], h2 = chi[2 * k + 1];
        unwrap_arcs(l2, h2);
        l = make_uint4(min(l.x, l2.x), min(l.y, l2.y), min(l.z, l2.z), max(l.w, l2.w));
        h = make_uint4(max(h.x, h2.x), max(h.y, h2.y), max(h.z, h2.z), h.w + h2.w);
        if (cbox) {
            uint32_t b2 = cbox[2 * k + 1];
            b = min(b & 0xffffu, b2 & 0xffffu) | (max(b >> 16, b2 >> 16) << 16);
        }
    }
    plo[k] = l;
    phi[k] = h;
    if (cbox) pbox[k] = b;
}

// periodic gap (fixed point) between the arcs [a0,a1] and [b0,b1] of a circle
// of 2^32 (an arc may wrap, a0 > a1): 0 when they meet, else the shorter way
// round; all differences modulo 2^32
__device__ __forceinline__ unsigned long long axis_gap(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
    if (b0 - a0 <= a1 - a0 || a0 - b0 <= b1 - b0) return 0ull;
    const uint32_t g1 = b0 - a1, g2 = a0 - b1;
    return (unsigned long long)(g1 < g2 ? g1 : g2);
}

__device__ __forceinline__ unsigned long long box_gap2(uint4 alo, uint4 ahi, uint4 blo, uint4 bhi) {
    unsigned long long gx = axis_gap(alo.x, ahi.x, blo.x, bhi.x);
    unsigned long long gy = axis_gap(alo.y, ahi.y, blo.y, bhi.y);
    unsigned long long gz = axis_gap(alo.z, ahi.z, blo.z, bhi.z);
    return gx * gx + gy * gy + gz * gz;
}

// 32-ary view of the binary tile tree: 32-ary level L is binary level 5 L, and
// the children of node k are nodes 32 k .. 32 k + 31 one 32-ary level down.
constexpr int MAX_L32 = 8;
constexpr int LIST_WARPS = 4;
constexpr int STACK = 256;

struct Tree32 {
    int off[MAX_L32];
    int cnt[MAX_L32];
    int top;          // highest 32-ary level (at most 32 nodes)
};

// Warp-cooperative depth-first walk for tile I (one warp): every lane tests one
// child of the node being expanded; passing leaves (tiles) are emitted in
// ascending order, passing inner nodes pushed so that the lowest pops first.
// The reach of a node is max(Hmax_I, Hmax_node) (pair-set predicate).
template <bool WRITE>
__device__ uint32_t walk32(const Tree32 &T, const uint4 *__restrict__ lo, const uint4 *__restrict__ hi,
                           const uint32_t *__restrict__ nbox, uint32_t Ibox, uint4 Ilo, uint4 Ihi,
                           uint32_t *__restrict__ out, uint32_t lim, int *stL, int *stK, int lane) {
    const unsigned lt = lanemask_lt();
    const unsigned long long HI = Ilo.w;
    uint32_t count = 0;
    int sp = 0;
    int L = T.top + 1, k = 0;           // virtual root: its children are the top-level nodes
    for (;;) {
        const int cl = L - 1;
        const int c = k * 32 + lane;
        bool pass = false;
        if (c < T.cnt[cl]) {
            const uint4 nlo = lo[T.off[cl] + c], nhi = hi[T.off[cl] + c];
            unsigned long long R = HI > (unsigned long long)nlo.w ? HI : (unsigned long long)nlo.w;
            pass = box_gap2(Ilo, Ihi, nlo, nhi) < R * R &&
                   (!nbox || box_ranges_meet(Ibox, nbox[T.off[cl] + c]));
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        const int np = __popc(m);
        if (cl == 0) {
            if (WRITE && pass) {
                const uint32_t at = count + __popc(m & lt);
                if (at < lim) out[at] = (uint32_t)c;
            }
            count += np;
        } else if (np) {
            if (pass) {
                const int pos = sp + (np - 1 - __popc(m & lt));
                if (pos < STACK) { stL[pos] = cl; stK[pos] = c; }
            }
            sp += np;
        }
        __syncwarp();
        if (sp == 0) break;
        sp--;
        if (sp >= STACK) return 0xffffffffu;  // stack overflow: caller reports
        L = stL[sp];
        k = stK[sp];
        __syncwarp();
    }
    return count;
}

constexpr uint32_t LIST_BUF = 1024;   // tiles a warp keeps in shared memory

// One walk per tile into shared memory, then one allocation and a coalesced
// copy; a tile with more than LIST_BUF neighbours walks a second time
// straight into the allocated range.  act (may be null): the lists of the
// tiles act[0 .. count) only.
__global__ void __launch_bounds__(LIST_WARPS * 32) k_lists32(int count, const int32_t *__restrict__ act, Tree32 T,
                                                             const uint4 *__restrict__ lo,
                                                             const uint4 *__restrict__ hi,
                                                             const uint32_t *__restrict__ nbox,
                                                             uint2 *__restrict__ ofs, uint32_t *__restrict__ list,
                                                             long long cap, unsigned long long *counter) {
    __shared__ int stL[LIST_WARPS][STACK], stK[LIST_WARPS][STACK];
    __shared__ uint32_t buf[LIST_WARPS][LIST_BUF];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * LIST_WARPS + w;
    if (t >= count) return;
    const int I = act ? act[t] : t;
    const uint4 Ilo = lo[I], Ihi = hi[I];
    const uint32_t Ibox = nbox ? nbox[I] : 0u;
    uint32_t c = walk32<true>(T, lo, hi, nbox, Ibox, Ilo, Ihi, buf[w], LIST_BUF, stL[w], stK[w], lane);
    unsigned long long base = 0;
    if (c == 0xffffffffu) {
        if (lane == 0) {
            atomicAdd(counter, (unsigned long long)cap + 1ull);   // forces the overflow path
            ofs[I] = make_uint2(0u, 0u);
        }
        return;
    }
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)c);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)(base + c) <= cap) {
        __syncwarp();
        if (c <= LIST_BUF) {
            for (uint32_t k = lane; k < c; k += 32) list[base + k] = buf[w][k];
        } else {
            walk32<true>(T, lo, hi, nbox, Ibox, Ilo, Ihi, list + base, c, stL[w], stK[w], lane);
        }
        if (lane == 0) ofs[I] = make_uint2((uint32_t)base, c);
    } else if (lane == 0) {
        ofs[I] = make_uint2(0u, 0u);
    }
}

// ------------------------------------------------------------------ cell table

__device__ __forceinline__ int cell_level(unsigned long long hbits, int kmax) {
    float hmax = __uint_as_float((uint32_t)hbits);
    int e;
    float m = frexpf(hmax, &e);
    int k = (m == 0.5f) ? 1 - e : -e;
    return max(1, min(kmax, k));
}

__global__ void k_cell_start(int n, const uint32_t *__restrict__ keys, int kmax,
                             const unsigned long long *__restrict__ counters, int32_t *__restrict__ cs) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    int k = cell_level(counters[CNT_HMAX], kmax);
    int sh = 30 - 3 * k;
    long long ncell = 1ll << (3 * k);
    if (s > n) return;
    long long c = (s < n) ? (long long)(keys[s] >> sh) : ncell;
    long long cp = (s > 0) ? (long long)(keys[s - 1] >> sh) : -1;
    for (long long cc = cp + 1; cc <= c; cc++) cs[cc] = s;
}

// ------------------------------------------------------------------ drivers

static Tree32 tree32(const crk_ctx *ctx) {
    Tree32 T;
    int L = 0;
    for (; L < MAX_L32 && 5 * L < ctx->nlevels; L++) {
        T.off[L] = ctx->level_off[5 * L];
        T.cnt[L] = ctx->level_cnt[5 * L];
    }
    for (int k = L; k < MAX_L32; k++) {
        T.off[k] = 0;
        T.cnt[k] = 0;
    }
    T.top = L - 1;
    return T;
}

int rebuild_lists(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->ntiles == 0) return CRK_OK;
    Tree32 T = tree32(ctx);
    if (T.cnt[T.top] > 32) return crk_set_error(ctx, CRK_ECAPACITY, "tile tree too deep");
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_GLIST, 0, 2 * sizeof(unsigned long long), s));
    ctx->lists_valid = 0;
    const int count = ctx->act ? ctx->nact : ctx->ntiles;
    if (count == 0) return CRK_OK;
    k_lists32<<<grid_for(count, LIST_WARPS), LIST_WARPS * 32, 0, s>>>(
        count, ctx->act, T, ctx->node_lo, ctx->node_hi, ctx->nbox > 1 ? ctx->node_box : nullptr, ctx->uofs,
        ctx->ulist, ctx->cap_ulist, ctx->counters + CNT_ULIST);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "interaction lists");
    return CRK_OK;
}

// Tiles and tree from the sorted q4 (used again when only h changes).
int build_tree(crk_ctx *ctx, cudaStream_t s) {
    int n = ctx->n, nt = ctx->ntiles;
    if (nt == 0) return CRK_OK;
    const bool batched = ctx->nbox > 1;
    k_tiles<<<grid_for((long long)nt * 32, 256), 256, 0, s>>>(n, nt, ctx->q4, ctx->node_lo, ctx->node_hi,
                                                               batched ? ctx->sbox : nullptr, ctx->node_box);
    ++ctx->launches;
    for (int L = 1; L < ctx->nlevels; L++) {
        int pc = ctx->level_cnt[L];
        k_tree_level<<<grid_for(pc, 256), 256, 0, s>>>(ctx->node_lo + ctx->level_off[L - 1],
                                                         ctx->node_hi + ctx->level_off[L - 1],
                                                         ctx->level_cnt[L - 1],
                                                         ctx->node_lo + ctx->level_off[L],
                                                         ctx->node_hi + ctx->level_off[L], pc,
                                                         batched ? ctx->node_box + ctx->level_off[L - 1] : nullptr,
                                                         batched ? ctx->node_box + ctx->level_off[L] : nullptr);
        ++ctx->launches;
    }
    CRK_LAUNCH_CHECK(ctx, "tile tree");
    return CRK_OK;
}

// Bin the n records pos[t] (float4 x,y,z,h) of some input order; base_perm maps
// that order to caller indices (NULL = identity).  After the call idx_a holds,
// for every new sorted slot, its index in the input order.
__global__ void k_gather_u32(int n, const int32_t *__restrict__ idx, const uint32_t *__restrict__ in,
                             uint32_t *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = in[idx[s]];
}

int build_cells_sorted(crk_ctx *ctx, int n, const float4 *pos, const int32_t *base_perm, cudaStream_t s,
                       const int32_t *box_of_input) {
    int rc = crk_ensure_particles(ctx, n);
    if (rc) return rc;
    if (!box_of_input) ctx->nbox = 0;   // a build without boxes is one box
    ctx->n = n;
    ctx->ntiles = (n + TILE - 1) / TILE;
    int L = 0, c = ctx->ntiles, off = 0;
    while (c > 0 && L < MAX_LEVELS) {
        ctx->level_off[L] = off;
        ctx->level_cnt[L] = c;
        off += c;
        L++;
        if (c == 1) break;
        c = (c + 1) / 2;
    }
    ctx->nlevels = L;
    ctx->built = 0;
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_ERR_INPUT, 0, 2 * sizeof(unsigned long long), s));
    if (n == 0) {
        ctx->built = 1;
        return CRK_OK;
    }
    uint4 *q_tmp = ctx->q_tmp;
    float *h_tmp = ctx->h_tmp;
    prof_begin(ctx, PROF_BUILD, s);
    k_keys<<<grid_for(n, 256), 256, 0, s>>>(n, pos, ctx->key_a, ctx->idx_a, q_tmp, h_tmp, ctx->counters,
                                            ctx->p.tile_order == 1);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "keys");
    if (box_of_input && ctx->p.tile_order == 2)
        return crk_set_error(ctx, CRK_EINVAL, "the bisection order covers one box (tile_order 0 or 1 for batches)");
    if (box_of_input) {
        // batched boxes: stable sort by Morton key, then stable sort by box,
        // which leaves the order box-major and Morton within each box
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->mkey, ctx->key_a, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        rc = radix_sort(ctx, n, 30, s);
        if (rc) return rc;
        k_gather_u32<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->idx_a, reinterpret_cast<const uint32_t *>(box_of_input),
                                                      ctx->key_a);
        ++ctx->launches;
        rc = radix_sort(ctx, n, ctx->nbox <= 256 ? 8 : 16, s);
        if (rc) return rc;
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->sbox, ctx->key_a, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        k_gather_u32<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->idx_a, ctx->mkey, ctx->keys);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "box sort");
    } else {
        rc = radix_sort(ctx, n, 30, s);
        if (rc) return rc;
        // sorted keys (read by the chaining-mesh table, which only the Morton order has)
        CRK_CUDA(ctx, cudaMemcpyAsync(ctx->keys, ctx->key_a, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        if (ctx->p.tile_order == 2) {
            rc = rcb_refine(ctx, n, s);
            if (rc) return rc;
        }
    }
    k_gather_sorted<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->idx_a, q_tmp, h_tmp, base_perm, ctx->q4,
                                                     ctx->hs, ctx->idx_b);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "gather sorted");
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->perm, ctx->idx_b, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    if (!box_of_input && ctx->p.tile_order == 0) {   // the chaining-mesh table: one box, Morton order
        k_cell_start<<<grid_for(n + 1, 256), 256, 0, s>>>(n, ctx->keys, ctx->p.kmax, ctx->counters,
                                                          ctx->cell_start);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "cell table");
    }
    rc = build_tree(ctx, s);
    if (rc) return rc;
    rc = rebuild_lists(ctx, s);
    if (rc) return rc;
    prof_end(ctx, s);
    ctx->built = 1;
    return CRK_OK;
}

__global__ void k_len_keys(int nt, const uint32_t *__restrict__ len, uint32_t *__restrict__ key,
                           int32_t *__restrict__ idx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    key[t] = 0xffffu - min(len[t], 0xffffu);
    idx[t] = t;
}

// ctx->tile_order = tiles sorted by decreasing pair-set list length (stable:
// equal lengths keep Morton order), for the longest-first pass variants.
int tile_order_by_length(crk_ctx *ctx, cudaStream_t s) {
    const int nt = ctx->ntiles;
    if (nt > ctx->cap_order) {
        if (ctx->tile_order) cudaFree(ctx->tile_order);
        ctx->tile_order = nullptr;
        ctx->cap_order = 0;
        CRK_CUDA(ctx, cudaMalloc((void **)&ctx->tile_order, sizeof(int32_t) * (size_t)nt));
        ctx->cap_order = nt;
    }
    k_len_keys<<<grid_for(nt, 256), 256, 0, s>>>(nt, ctx->len_u, ctx->key_a, ctx->idx_a);
    ++ctx->launches;
    int rc = radix_sort(ctx, nt, 16, s);
    if (rc) return rc;
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->tile_order, ctx->idx_a, sizeof(int32_t) * (size_t)nt,
                                  cudaMemcpyDeviceToDevice, s));
    CRK_LAUNCH_CHECK(ctx, "tile order");
    return CRK_OK;
}

int cell_level_host(const crk_ctx *ctx) {
    uint32_t bits = (uint32_t)ctx->h_counters[CNT_HMAX];
    float hmax;
    memcpy(&hmax, &bits, sizeof(float));
    int e;
    float m = frexpf(hmax, &e);
    int k = (m == 0.5f) ? 1 - e : -e;
    return k < 1 ? 1 : (k > ctx->p.kmax ? ctx->p.kmax : k);
}

// Read the counters after a build; grow and redo the lists on overflow.
int finish_build(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->graph_mode) return CRK_OK;   // captured step: checked after the replay
    int rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    if (ctx->h_counters[CNT_ERR_INPUT])
        return crk_set_error(ctx, CRK_EINVAL, "%llu particle records have coordinates outside [0,1) "
                             "or h outside (0, 1/3)", ctx->h_counters[CNT_ERR_INPUT]);
    long long ng = 0, nu = (long long)ctx->h_counters[CNT_ULIST];
    if (nu > ctx->cap_ulist) {
        rc = crk_ensure_lists(ctx, 0, nu + nu / 4 + 1024);
        if (rc) return rc;
        rc = rebuild_lists(ctx, s);
        if (rc) return rc;
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        nu = (long long)ctx->h_counters[CNT_ULIST];
        if (nu > ctx->cap_ulist)
            return crk_set_error(ctx, CRK_ECAPACITY, "interaction lists overflow after growth");
    }
    ctx->glist_total = ng;
    ctx->ulist_total = nu;
    ctx->cell_k = cell_level_host(ctx);
    return CRK_OK;
}

}  // namespace crk
