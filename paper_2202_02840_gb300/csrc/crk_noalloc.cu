// crk_noalloc.cu -- particle volumes (P1) for callers that cannot allocate
// device memory.
//
// Some callers own every byte of device memory through their own allocator
// (a simulation that pre-reserves the GPU for its particle arrays and hands
// out sub-buffers), or must not call cudaMalloc/cudaFree at all because
// those calls can synchronise the whole device in the middle of their work.
// This entry point serves them: all of its scratch (sort keys and indices,
// sorted records, tiles, the tile tree, interaction lists, histograms and
// counters) lives in one file-scope __device__ array of fixed size, so a call
// allocates nothing.  The caller still passes its inputs and outputs.
//
// The array is shared by every call in the process and keeps the contents of
// the last call; each call clears what must start at zero.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array and must be serialised by the caller.
#include "crk_internal.cuh"

#include <atomic>

namespace {

constexpr int NMAX = CRK_NOALLOC_MAX_N;
// whole tiles only: n = NMAX must not make a tile past the per-tile sub-buffers
static_assert(NMAX % crk::TILE == 0, "CRK_NOALLOC_MAX_N must be a multiple of the 32-particle tile");
constexpr int TMAX = NMAX / crk::TILE;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t key_a, key_b, idx_a, idx_b, keys, perm, q_tmp, q4, h_tmp, hs, V, Nn, qV, cnt_g, cnt_u;
    size_t nlo, nhi, uofs, ulist, len_g, len_u, hist, scan, cells, counters, total;
};

constexpr Layout make_layout() {
    Layout L{};
    size_t o = 0;
    L.key_a = o;    o = al(o + 4ull * NMAX);
    L.key_b = o;    o = al(o + 4ull * NMAX);
    L.idx_a = o;    o = al(o + 4ull * NMAX);
    L.idx_b = o;    o = al(o + 4ull * NMAX);
    L.keys = o;     o = al(o + 4ull * NMAX);
    L.perm = o;     o = al(o + 4ull * NMAX);
    L.q_tmp = o;    o = al(o + 16ull * NMAX);
    L.q4 = o;       o = al(o + 16ull * NMAX);
    L.h_tmp = o;    o = al(o + 4ull * NMAX);
    L.hs = o;       o = al(o + 4ull * NMAX);
    L.V = o;        o = al(o + 4ull * NMAX);
    L.Nn = o;       o = al(o + 4ull * NMAX);
    L.qV = o;       o = al(o + 16ull * NMAX);
    L.cnt_g = o;    o = al(o + 4ull * NMAX);
    L.cnt_u = o;    o = al(o + 4ull * NMAX);
    L.nlo = o;      o = al(o + 16ull * (2 * TMAX + crk::MAX_LEVELS));
    L.nhi = o;      o = al(o + 16ull * (2 * TMAX + crk::MAX_LEVELS));
    L.uofs = o;     o = al(o + 8ull * TMAX);
    L.ulist = o;    o = al(o + 4ull * TMAX * TMAX);   // every tile may neighbour every tile
    L.len_g = o;    o = al(o + 4ull * TMAX);
    L.len_u = o;    o = al(o + 4ull * TMAX);
    L.hist = o;     o = al(o + 4ull * 256 * ((NMAX + 4095) / 4096));
    L.scan = o;     o = al(o + 4ull * (2 * 4096 + 64));
    L.cells = o;    o = al(o + 4ull * 9);              // chaining-mesh table at level 1
    L.counters = o; o = al(o + 8ull * crk::CNT_COUNT);
    L.total = o;
    return L;
}

constexpr Layout LAY = make_layout();
// the size the header documents (about 3.0 MB)
static_assert(LAY.total <= 3200000, "the allocation-free scratch outgrew its documented size");

}  // namespace

// The scratch of every call (about 3.0 MB for NMAX = 16384).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LAY.total];

// Device address of g_noalloc_scratch, resolved once per device.  Host
// threads making their first call at the same time may both resolve it; they
// store the same address, and the atomic makes that race-free.
static std::atomic<void *> g_scratch_addr[64];

extern "C" int crk_volumes_noalloc(int n, const float *pos_h, float *V, float *Nngb, void *stream) {
    if (n < 0 || n > NMAX) return CRK_EINVAL;
    if (n > 0 && (!pos_h || !V)) return CRK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CRK_ECUDA;
    if (dev < 0 || dev >= 64) return CRK_EINVAL;
    void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return CRK_ECUDA;
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    unsigned char *b = (unsigned char *)addr;
    cudaStream_t s = (cudaStream_t)stream;

    crk_ctx ctx;                      // host stack: no allocation anywhere
    crk_default_params(&ctx.p);
    ctx.p.kmax = 1;
    ctx.volumes_only = 1;             // P1 only: the walk writes no neighbour lists
    ctx.err[0] = 0;
    ctx.device = dev;
    ctx.key_a = (uint32_t *)(b + LAY.key_a);
    ctx.key_b = (uint32_t *)(b + LAY.key_b);
    ctx.idx_a = (int32_t *)(b + LAY.idx_a);
    ctx.idx_b = (int32_t *)(b + LAY.idx_b);
    ctx.keys = (uint32_t *)(b + LAY.keys);
    ctx.perm = (int32_t *)(b + LAY.perm);
    ctx.q_tmp = (uint4 *)(b + LAY.q_tmp);
    ctx.q4 = (uint4 *)(b + LAY.q4);
    ctx.h_tmp = (float *)(b + LAY.h_tmp);
    ctx.hs = (float *)(b + LAY.hs);
    ctx.V = (float *)(b + LAY.V);
    ctx.Nn = (float *)(b + LAY.Nn);
    ctx.qV = (uint4 *)(b + LAY.qV);
    ctx.cnt_g = (int32_t *)(b + LAY.cnt_g);
    ctx.cnt_u = (int32_t *)(b + LAY.cnt_u);
    ctx.node_lo = (uint4 *)(b + LAY.nlo);
    ctx.node_hi = (uint4 *)(b + LAY.nhi);
    ctx.uofs = (uint2 *)(b + LAY.uofs);
    ctx.ulist = (uint32_t *)(b + LAY.ulist);
    ctx.len_g = (uint32_t *)(b + LAY.len_g);
    ctx.len_u = (uint32_t *)(b + LAY.len_u);
    ctx.hist = (uint32_t *)(b + LAY.hist);
    ctx.scan_tmp = (uint32_t *)(b + LAY.scan);
    ctx.cell_start = (int32_t *)(b + LAY.cells);
    ctx.counters = (unsigned long long *)(b + LAY.counters);
    ctx.cap_n = NMAX;
    ctx.cap_tiles = TMAX;
    ctx.cap_nodes = 2 * TMAX + crk::MAX_LEVELS;
    ctx.cap_hist = 256 * ((NMAX + 4095) / 4096);
    ctx.cap_ulist = (long long)TMAX * TMAX;

    if (cudaMemsetAsync(ctx.counters, 0, sizeof(unsigned long long) * crk::CNT_COUNT, s) != cudaSuccess)
        return CRK_ECUDA;
    int rc = crk::build_cells_sorted(&ctx, n, (const float4 *)pos_h, nullptr, s);
    if (rc) return rc;
    if (n == 0) return CRK_OK;
    unsigned long long hc[crk::CNT_COUNT];
    if (cudaMemcpyAsync(hc, ctx.counters, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRK_ECUDA;
    if (hc[crk::CNT_ERR_INPUT]) return CRK_EINVAL;
    if ((long long)hc[crk::CNT_ULIST] > ctx.cap_ulist) return CRK_ECAPACITY;
    rc = crk::run_volumes(&ctx, s);
    if (!rc) rc = crk::scatter_rows(&ctx, ctx.V, V, 1, s);
    if (!rc && Nngb) rc = crk::scatter_rows(&ctx, ctx.Nn, Nngb, 1, s);
    // Every buffer above was sized for NMAX, so nothing may have been grown;
    // a later change to the build or the pass that did grow one would have
    // swapped in library-allocated memory: report it rather than return.
    if (!rc && ctx.alloc_gen != 0) return CRK_ESTATE;
    return rc;
}
