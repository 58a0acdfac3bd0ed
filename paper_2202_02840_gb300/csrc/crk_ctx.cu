// crk_ctx.cu -- engine lifecycle, device memory, caller-order packing and the
// C-ABI entry points of the individual passes (declared in include/crk.h).
#include "crk_internal.cuh"

#include <new>
#include <stdlib.h>
#include <string.h>

using namespace crk;

// ------------------------------------------------------------------ errors

int crk_set_error(crk_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int crk_check_cuda(crk_ctx *ctx, cudaError_t e, const char *what) {
    int code = (e == cudaErrorMemoryAllocation) ? CRK_ENOMEM : CRK_ECUDA;
    return crk_set_error(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ memory

template <typename T>
static int dalloc(crk_ctx *ctx, T **p, size_t count) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (ctx) ctx->alloc_gen++;   // captured graphs hold the old addresses
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return crk_check_cuda(ctx, e, "cudaMalloc");
    }
    return CRK_OK;
}

template <typename T>
static void dfree(T **p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

int crk_ensure_particles(crk_ctx *ctx, int n) {
    if (n <= ctx->cap_n && ctx->q4) return CRK_OK;
    int cap = n < 4096 ? 4096 : n + n / 8;
    int tiles = (cap + TILE - 1) / TILE;
    int nb = (cap + 4095) / 4096;
    int rc = 0;
    rc |= dalloc(ctx, &ctx->key_a, cap);
    rc |= dalloc(ctx, &ctx->key_b, cap);
    rc |= dalloc(ctx, &ctx->idx_a, cap);
    rc |= dalloc(ctx, &ctx->idx_b, cap);
    rc |= dalloc(ctx, &ctx->keys, cap);
    rc |= dalloc(ctx, &ctx->perm, cap);
    rc |= dalloc(ctx, &ctx->q4, cap);
    rc |= dalloc(ctx, &ctx->hs, cap);
    rc |= dalloc(ctx, &ctx->V, cap);
    rc |= dalloc(ctx, &ctx->Nn, cap);
    rc |= dalloc(ctx, &ctx->vel, cap);
    rc |= dalloc(ctx, &ctx->mass, cap);
    rc |= dalloc(ctx, &ctx->corr, cap);
    rc |= dalloc(ctx, &ctx->gv, cap);
    rc |= dalloc(ctx, &ctx->acc, cap);
    rc |= dalloc(ctx, &ctx->vq, cap);
    rc |= dalloc(ctx, &ctx->vb, cap);
    rc |= dalloc(ctx, &ctx->va, cap);
    rc |= dalloc(ctx, &ctx->du, cap);
    rc |= dalloc(ctx, &ctx->st_pos, cap);
    rc |= dalloc(ctx, &ctx->st_vel, cap);
    rc |= dalloc(ctx, &ctx->st_half, cap);
    rc |= dalloc(ctx, &ctx->st_tmp, cap);
    rc |= dalloc(ctx, &ctx->st_tmp1, cap);
    rc |= dalloc(ctx, &ctx->q_tmp, cap);
    rc |= dalloc(ctx, &ctx->h_tmp, cap);
    rc |= dalloc(ctx, &ctx->flags, cap);
    rc |= dalloc(ctx, &ctx->d_dt, cap);
    rc |= dalloc(ctx, &ctx->rho, cap);
    rc |= dalloc(ctx, &ctx->uofs, tiles);
    rc |= dalloc(ctx, &ctx->qV, cap);
    rc |= dalloc(ctx, &ctx->cnt_g, cap);
    rc |= dalloc(ctx, &ctx->cnt_u, cap);
    rc |= dalloc(ctx, &ctx->lowc, cap);
    rc |= dalloc(ctx, &ctx->po_self, tiles);
    rc |= dalloc(ctx, &ctx->po_tofs, tiles);
    rc |= dalloc(ctx, &ctx->len_g, tiles);
    rc |= dalloc(ctx, &ctx->len_u, tiles);
    rc |= dalloc(ctx, &ctx->tbase, tiles);
    rc |= dalloc(ctx, &ctx->frec, 10 * (size_t)cap);
    rc |= dalloc(ctx, &ctx->sfun, cap);
    rc |= dalloc(ctx, &ctx->sig, cap);
    rc |= dalloc(ctx, &ctx->sig2, 2 * (size_t)cap);   // two kicks' sums side by side
    rc |= dalloc(ctx, &ctx->du_next, cap);
    rc |= dalloc(ctx, &ctx->node_lo, 2 * (size_t)tiles + MAX_LEVELS);
    rc |= dalloc(ctx, &ctx->node_hi, 2 * (size_t)tiles + MAX_LEVELS);
    rc |= dalloc(ctx, &ctx->hist, 256 * (size_t)nb);
    rc |= dalloc(ctx, &ctx->d_red, 4096 * 8);
    if (rc) {
        ctx->cap_n = 0;
        return crk_set_error(ctx, CRK_ENOMEM, "cannot allocate buffers for %d particles", n);
    }
    ctx->cap_n = cap;
    ctx->cap_tiles = tiles;
    ctx->cap_nodes = 2 * tiles + MAX_LEVELS;
    ctx->cap_hist = 256 * nb;
    ctx->rates_valid = 0;
    ctx->lists_valid = 0;
    long long want = (long long)tiles * 48;
    if (ctx->cap_ulist < want) return crk_ensure_lists(ctx, 0, want);
    return CRK_OK;
}

// List entries (fixed layout, n_ent) and stored forces (compact, n_force);
// a negative size leaves that buffer as it is.
int crk_ensure_entries(crk_ctx *ctx, long long n_ent, long long n_force) {
    if (n_ent > ctx->ent_cap || !ctx->ent) {
        long long cap = n_ent < 4096 ? 4096 : n_ent;
        if (dalloc(ctx, &ctx->ent, (size_t)cap)) {
            ctx->ent_cap = 0;
            return crk_set_error(ctx, CRK_ENOMEM, "cannot allocate %lld neighbour-list entries", cap);
        }
        ctx->ent_cap = cap;
    }
    if (n_force > ctx->f_cap || !ctx->Fst) {
        long long cap = n_force + n_force / 5 + 4096;
        if (dalloc(ctx, &ctx->Fst, (size_t)cap)) {
            ctx->f_cap = 0;
            return crk_set_error(ctx, CRK_ENOMEM, "cannot allocate %lld stored pair forces", cap);
        }
        ctx->f_cap = cap;
    }
    return CRK_OK;
}

// Grow the stored-force buffer to n_force entries, keeping its contents (the
// forces of the last evaluation, which the next step's first kick reads).
int crk_grow_forces_keep(crk_ctx *ctx, long long n_force) {
    if (n_force <= ctx->f_cap && ctx->Fst) return CRK_OK;
    float4 *nb = nullptr;
    cudaError_t e = cudaMalloc((void **)&nb, sizeof(float4) * (size_t)n_force);
    if (e != cudaSuccess) return crk_check_cuda(ctx, e, "cudaMalloc");
    if (ctx->Fst && ctx->f_cap > 0) {
        e = cudaMemcpy(nb, ctx->Fst, sizeof(float4) * (size_t)ctx->f_cap, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            cudaFree(nb);
            return crk_check_cuda(ctx, e, "cudaMemcpy");
        }
        cudaFree(ctx->Fst);
    }
    ctx->Fst = nb;
    ctx->f_cap = n_force;
    ctx->alloc_gen++;
    return CRK_OK;
}

// Arrays of the pair-once form, sized with the tile lists: per tile-list
// entry the reverse index, a copy of the entry (the tile lists the pass ran
// with, which P5 reads after the lists may have been refitted), and 32 lanes
// of j-side sums.  Sized on first use, so that contexts that never evaluate
// forces do not hold them; growing keeps the reverse index and the copy (the
// next kick's P5 reads them), and a captured step finds them sized before the
// capture.
template <typename T>
static int grow_keep(crk_ctx *ctx, T **p, long long old_n, long long new_n) {
    T *nb = nullptr;
    cudaError_t e = cudaMalloc((void **)&nb, sizeof(T) * (size_t)new_n);
    if (e != cudaSuccess) return crk_check_cuda(ctx, e, "cudaMalloc");
    if (*p && old_n > 0) {
        e = cudaMemcpy(nb, *p, sizeof(T) * (size_t)old_n, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) {
            cudaFree(nb);
            return crk_check_cuda(ctx, e, "cudaMemcpy");
        }
    }
    if (*p) cudaFree(*p);
    *p = nb;
    ctx->alloc_gen++;
    return CRK_OK;
}

int crk_ensure_pair_once(crk_ctx *ctx) {
    const long long want = ctx->cap_ulist;
    if (ctx->po_cap >= want && ctx->po_rev) return CRK_OK;
    if (ctx->graph_mode) return crk_set_error(ctx, CRK_ESTATE, "pair-once arrays grow during a capture");
    int rc = grow_keep(ctx, &ctx->po_rev, ctx->po_cap, want);
    if (!rc) rc = grow_keep(ctx, &ctx->po_tlist, ctx->po_cap, want);
    if (!rc) rc = dalloc(ctx, &ctx->po_rowA, 32 * (size_t)want);
    if (!rc) rc = dalloc(ctx, &ctx->po_rowB, 32 * (size_t)want);
    if (rc) {
        ctx->po_cap = 0;
        return crk_set_error(ctx, CRK_ENOMEM, "cannot allocate pair-once sums for %lld tile pairs", want);
    }
    ctx->po_cap = want;
    return CRK_OK;
}

int crk_ensure_lists(crk_ctx *ctx, long long ng, long long nu) {
    if (ng > 0xffffffffll || nu > 0xffffffffll)
        return crk_set_error(ctx, CRK_ECAPACITY, "interaction lists beyond 2^32 entries");
    int rc = 0;
    if (ng > ctx->cap_glist) {
        rc |= dalloc(ctx, &ctx->glist, (size_t)ng);
        ctx->cap_glist = rc ? 0 : ng;
    }
    if (nu > ctx->cap_ulist) {
        rc |= dalloc(ctx, &ctx->ulist, (size_t)nu);
        ctx->cap_ulist = rc ? 0 : nu;
    }
    if (rc) return crk_set_error(ctx, CRK_ENOMEM, "cannot allocate interaction lists");
    return CRK_OK;
}

int crk_sync_counters(crk_ctx *ctx, cudaStream_t s) {
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->h_counters, ctx->counters, CNT_COUNT * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s));
    CRK_CUDA(ctx, cudaStreamSynchronize(s));
    if (ctx->h_counters[CNT_TMA_ERR])   // a TMA-fed pass timed out on its copies (sticky)
        return crk_set_error(ctx, CRK_ECUDA, "a TMA-fed pass gave up waiting on its copies");
    if (ctx->h_counters[CNT_PO_MISS])   // the tile lists were not symmetric (sticky)
        return crk_set_error(ctx, CRK_ESTATE, "pair-once: %llu tile pairs without their reverse",
                             ctx->h_counters[CNT_PO_MISS]);
    return CRK_OK;
}

// ------------------------------------------------------------------ pack / unpack kernels

__global__ void k_gather_rows(long long total, int w, const int32_t *__restrict__ perm,
                              const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    long long s = t / w;
    int c = (int)(t - s * w);
    out[t] = in[(long long)perm[s] * w + c];
}

__global__ void k_scatter_rows(long long total, int w, const int32_t *__restrict__ perm,
                               const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    long long s = t / w;
    int c = (int)(t - s * w);
    out[(long long)perm[s] * w + c] = in[t];
}

// caller-order (A, B, gA, gB) -> sorted CorrRec
__global__ void k_pack_corr(int n, const int32_t *__restrict__ perm, const float *__restrict__ A,
                            const float *__restrict__ B, const float *__restrict__ gA,
                            const float *__restrict__ gB, CorrRec *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    long long i = perm[s];
    const float *b = B + 3 * i, *ga = gA + 3 * i, *gb = gB + 9 * i;
    CorrRec c;
    c.c0 = make_float4(A[i], b[0], b[1], b[2]);
    c.c1 = make_float4(ga[0], ga[1], ga[2], gb[0]);
    c.c2 = make_float4(gb[1], gb[2], gb[3], gb[4]);
    c.c3 = make_float4(gb[5], gb[6], gb[7], gb[8]);
    out[s] = c;
}

__global__ void k_unpack_corr(int n, const int32_t *__restrict__ perm, const CorrRec *__restrict__ in,
                              float *__restrict__ A, float *__restrict__ B, float *__restrict__ gA,
                              float *__restrict__ gB) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    long long i = perm[s];
    CorrRec c = in[s];
    A[i] = c.c0.x;
    float *b = B + 3 * i, *ga = gA + 3 * i, *gb = gB + 9 * i;
    b[0] = c.c0.y; b[1] = c.c0.z; b[2] = c.c0.w;
    ga[0] = c.c1.x; ga[1] = c.c1.y; ga[2] = c.c1.z;
    gb[0] = c.c1.w; gb[1] = c.c2.x; gb[2] = c.c2.y; gb[3] = c.c2.z; gb[4] = c.c2.w;
    gb[5] = c.c3.x; gb[6] = c.c3.y; gb[7] = c.c3.z; gb[8] = c.c3.w;
}

__global__ void k_pack_gv(int n, const int32_t *__restrict__ perm, const float *__restrict__ g,
                          GvRec *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float *a = g + 9 * (long long)perm[s];
    GvRec r;
    r.g0 = make_float4(a[0], a[1], a[2], a[3]);
    r.g1 = make_float4(a[4], a[5], a[6], a[7]);
    r.g2 = make_float4(a[8], 0.f, 0.f, 0.f);
    out[s] = r;
}

__global__ void k_unpack_gv(int n, const int32_t *__restrict__ perm, const GvRec *__restrict__ in,
                            float *__restrict__ g) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float *a = g + 9 * (long long)perm[s];
    GvRec r = in[s];
    a[0] = r.g0.x; a[1] = r.g0.y; a[2] = r.g0.z; a[3] = r.g0.w;
    a[4] = r.g1.x; a[5] = r.g1.y; a[6] = r.g1.z; a[7] = r.g1.w;
    a[8] = r.g2.x;
}

// caller float[3n] -> sorted float4 (w = 0)
__global__ void k_pack_v3(int n, const int32_t *__restrict__ perm, const float *__restrict__ v,
                          float4 *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float *a = v + 3 * (long long)perm[s];
    out[s] = make_float4(a[0], a[1], a[2], 0.f);
}

// sorted (ax, ay, az, dudt) and (vsig, qmax) -> caller arrays
__global__ void k_unpack_forces(int n, const int32_t *__restrict__ perm, const float4 *__restrict__ acc,
                                const float2 *__restrict__ vq, float *__restrict__ accel,
                                float *__restrict__ dudt, float *__restrict__ vsig, float *__restrict__ qmax) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    long long i = perm[s];
    float4 a = acc[s];
    accel[3 * i] = a.x;
    accel[3 * i + 1] = a.y;
    accel[3 * i + 2] = a.z;
    if (dudt) dudt[i] = a.w;
    float2 q = vq[s];
    if (vsig) vsig[i] = q.x;
    if (qmax) qmax[i] = q.y;
}

// (q, V) records of the gather passes from the sorted V
__global__ void k_make_qV(int n, const uint4 *__restrict__ q4, const float *__restrict__ V, uint4 *__restrict__ qV) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint4 q = q4[s];
    qV[s] = make_uint4(q.x, q.y, q.z, __float_as_uint(V[s]));
}

namespace crk {
int gather_rows(crk_ctx *ctx, const void *in, void *out, int w, cudaStream_t s) {
    long long total = (long long)ctx->n * w;
    if (total == 0) return CRK_OK;
    k_gather_rows<<<grid_for(total, 256), 256, 0, s>>>(total, w, ctx->perm, (const uint32_t *)in, (uint32_t *)out);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "gather rows");
    return CRK_OK;
}
int scatter_rows(crk_ctx *ctx, const void *in, void *out, int w, cudaStream_t s) {
    long long total = (long long)ctx->n * w;
    if (total == 0) return CRK_OK;
    k_scatter_rows<<<grid_for(total, 256), 256, 0, s>>>(total, w, ctx->perm, (const uint32_t *)in, (uint32_t *)out);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "scatter rows");
    return CRK_OK;
}
}  // namespace crk

// ------------------------------------------------------------------ pass timing

namespace crk {
void prof_begin(crk_ctx *ctx, int id, cudaStream_t s) {
    if (!ctx->prof_on || ctx->prof_n >= ctx->prof_cap) return;
    ctx->prof_id[ctx->prof_n] = id;
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], s);
}
void prof_end(crk_ctx *ctx, cudaStream_t s) {
    if (!ctx->prof_on || ctx->prof_n >= ctx->prof_cap) return;
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], s);
    ctx->prof_n++;
}
}  // namespace crk

static void prof_free(crk_ctx *ctx) {
    if (ctx->prof_ev) {
        for (int k = 0; k < 2 * ctx->prof_cap; k++) cudaEventDestroy(ctx->prof_ev[k]);
        free(ctx->prof_ev);
        free(ctx->prof_id);
    }
    ctx->prof_ev = nullptr;
    ctx->prof_id = nullptr;
    ctx->prof_cap = 0;
}

extern "C" int crk_autotune(crk_ctx *ctx, int enable) {
    if (!ctx) return CRK_EINVAL;
    if (enable && !ctx->tune_ev[0]) {
        if (cudaEventCreate(&ctx->tune_ev[0]) != cudaSuccess || cudaEventCreate(&ctx->tune_ev[1]) != cudaSuccess)
            return crk_set_error(ctx, CRK_ECUDA, "cudaEventCreate");
    }
    ctx->tune_on = enable ? 1 : 0;
    if (enable)
        for (int k = 0; k < 16; k++) ctx->tune_done[k] = 0;
    return CRK_OK;
}

extern "C" int crk_tuning(crk_ctx *ctx, int *variant, float *ms) {
    if (!ctx) return CRK_EINVAL;
    for (int k = 0; k < CRK_PROF_NPASS; k++) {
        if (variant) variant[k] = ctx->tune_done[k] ? ctx->tune_choice[k] : -1;
        if (ms) ms[k] = ctx->tune_done[k] ? ctx->tune_ms[k] : 0.f;
    }
    return CRK_OK;
}

extern "C" int crk_tune_set(crk_ctx *ctx, int pass, int variant) {
    if (!ctx) return CRK_EINVAL;
    const bool list_pass = pass == PROF_P1 || pass == PROF_P2 || pass == PROF_P3 || pass == PROF_P4 ||
                           pass == PROF_P5 || pass == PROF_DENS;
    if (!list_pass || variant < -1 || variant >= NVAR)
        return crk_set_error(ctx, CRK_EINVAL, "crk_tune_set: no pass %d variant %d", pass, variant);
    const int slots[2] = {pass, pass == PROF_P5 ? TUNE_P5_DUAL : pass};
    for (int k : slots) {
        ctx->tune_choice[k] = variant;
        ctx->tune_done[k] = 1;
        ctx->tune_ms[k] = 0.f;
    }
    return CRK_OK;
}

extern "C" int crk_profile(crk_ctx *ctx, int enable) {
    if (!ctx) return CRK_EINVAL;
    if (enable && !ctx->prof_ev) {
        int cap = 4096;
        ctx->prof_ev = (cudaEvent_t *)calloc(2 * (size_t)cap, sizeof(cudaEvent_t));
        ctx->prof_id = (int *)calloc((size_t)cap, sizeof(int));
        if (!ctx->prof_ev || !ctx->prof_id) {
            prof_free(ctx);
            return crk_set_error(ctx, CRK_ENOMEM, "profile buffers");
        }
        for (int k = 0; k < 2 * cap; k++) {
            if (cudaEventCreate(&ctx->prof_ev[k]) != cudaSuccess) {
                ctx->prof_cap = k / 2;
                prof_free(ctx);
                return crk_set_error(ctx, CRK_ECUDA, "cudaEventCreate");
            }
            ctx->prof_cap = (k + 1) / 2;
        }
        ctx->prof_cap = cap;
    }
    ctx->prof_on = enable ? 1 : 0;
    if (enable) ctx->prof_n = 0;
    return CRK_OK;
}

extern "C" int crk_profile_read(crk_ctx *ctx, double *ms, long long *counts, long long *total_launches) {
    if (!ctx) return CRK_EINVAL;
    if (total_launches) *total_launches = ctx->launches;
    for (int k = 0; k < PROF_NPASS; k++) {
        if (ms) ms[k] = 0.0;
        if (counts) counts[k] = 0;
    }
    for (int r = 0; r < ctx->prof_n; r++) {
        CRK_CUDA(ctx, cudaEventSynchronize(ctx->prof_ev[2 * r + 1]));
        float t = 0.f;
        CRK_CUDA(ctx, cudaEventElapsedTime(&t, ctx->prof_ev[2 * r], ctx->prof_ev[2 * r + 1]));
        int id = ctx->prof_id[r];
        if (ms) ms[id] += t;
        if (counts) counts[id] += 1;
    }
    return CRK_OK;
}

// ------------------------------------------------------------------ lifecycle

extern "C" int crk_default_params(crk_params *p) {
    if (!p) return CRK_EINVAL;
    memset(p, 0, sizeof(*p));
    p->gamma = 5.0 / 3.0;
    p->n_h = 4.0;
    p->N_res = 268.0;
    p->C_l = 2.0;
    p->C_q = 1.0;
    p->eps = 0.1;
    p->eta_crit = 1.0 / 4.0;
    p->eta_fold = 0.2 / 4.0;
    p->C_cfl = 0.25;
    p->zeta = 4.0;
    p->h_min = 1e-6;
    p->h_max = 0.3;
    p->dt_max = 1.0;
    p->a = 1.0;
    p->adot = 0.0;
    p->precision = 1;
    p->kmax = 7;
    p->h_mode = 0;
    p->h_max_it = 50;
    p->h_tol = 1e-4f;
    p->rcb_leaf = 32;
    p->pair_form = 0;
    return CRK_OK;
}

extern "C" int crk_create(const crk_params *p, crk_ctx **out) {
    if (!out) return CRK_EINVAL;
    *out = nullptr;
    crk_params prm;
    if (p) prm = *p; else crk_default_params(&prm);
    if (!(prm.gamma > 1.0) || !(prm.n_h > 0) || !(prm.N_res > 0) || !(prm.eta_fold > 0) ||
        !(prm.h_max > 0 && prm.h_max < 1.0 / 3.0) || !(prm.h_min > 0 && prm.h_min < prm.h_max) ||
        prm.kmax < 1 || prm.kmax > 7 || prm.precision < 0 || prm.precision > 3 || !(prm.dt_max > 0) ||
        prm.tile_order < 0 || prm.tile_order > 2 || prm.density < 0 || prm.density > 1 || !(prm.a > 0.0) || !(prm.a < 1e30) ||
        !(prm.adot > -1e30 && prm.adot < 1e30) || prm.h_mode < 0 || prm.h_mode > 2 || prm.h_max_it < 1 ||
        !(prm.h_tol > 0.f) || (prm.rcb_leaf != 32 && prm.rcb_leaf != 128 && prm.rcb_leaf != 256) ||
        prm.pair_form < 0 || prm.pair_form > 1)
        return CRK_EINVAL;
    crk_ctx *ctx = new (std::nothrow) crk_ctx();
    if (!ctx) return CRK_ENOMEM;
    ctx->p = prm;
    ctx->err[0] = 0;
    memset(ctx->level_off, 0, sizeof(ctx->level_off));
    memset(ctx->level_cnt, 0, sizeof(ctx->level_cnt));
    int rc = CRK_OK;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        delete ctx;
        return CRK_ECUDA;
    }
    rc |= dalloc(ctx, &ctx->counters, CNT_COUNT);
    rc |= dalloc(ctx, &ctx->scan_tmp, 2 * 4096 + 64);
    rc |= dalloc(ctx, &ctx->cell_start, ((size_t)1 << (3 * prm.kmax)) + 1);
    rc |= dalloc(ctx, &ctx->d_scalars, 64);
    rc |= dalloc(ctx, &ctx->sm_next, 1024);
    if (!rc && cudaMallocHost((void **)&ctx->h_counters, CNT_COUNT * sizeof(unsigned long long)) != cudaSuccess)
        rc = CRK_ENOMEM;
    if (!rc && cudaMemset(ctx->counters, 0, CNT_COUNT * sizeof(unsigned long long)) != cudaSuccess) rc = CRK_ECUDA;
    if (rc) {
        crk_destroy(ctx);
        return CRK_ENOMEM;
    }
    *out = ctx;
    return CRK_OK;
}

extern "C" int crk_destroy(crk_ctx *ctx) {
    if (!ctx) return CRK_EINVAL;
    cudaDeviceSynchronize();
    dfree(&ctx->key_a); dfree(&ctx->key_b); dfree(&ctx->idx_a); dfree(&ctx->idx_b);
    dfree(&ctx->hist); dfree(&ctx->scan_tmp);
    dfree(&ctx->q4); dfree(&ctx->hs); dfree(&ctx->perm); dfree(&ctx->keys);
    dfree(&ctx->node_lo); dfree(&ctx->node_hi);
    dfree(&ctx->gofs); dfree(&ctx->uofs); dfree(&ctx->glist); dfree(&ctx->ulist);
    dfree(&ctx->qV); dfree(&ctx->cnt_g); dfree(&ctx->cnt_u); dfree(&ctx->len_g); dfree(&ctx->len_u);
    dfree(&ctx->tcap); dfree(&ctx->tbase); dfree(&ctx->ent); dfree(&ctx->Fst); dfree(&ctx->frec);
    dfree(&ctx->lowc); dfree(&ctx->po_self); dfree(&ctx->po_rev); dfree(&ctx->po_rowA); dfree(&ctx->po_rowB);
    dfree(&ctx->po_tofs); dfree(&ctx->po_tlist);
    dfree(&ctx->sfun); dfree(&ctx->sig); dfree(&ctx->sig2); dfree(&ctx->du_next);
    dfree(&ctx->cell_start); dfree(&ctx->counters);
    dfree(&ctx->V); dfree(&ctx->Nn); dfree(&ctx->vel); dfree(&ctx->mass);
    dfree(&ctx->corr); dfree(&ctx->gv); dfree(&ctx->acc); dfree(&ctx->vq);
    dfree(&ctx->vb); dfree(&ctx->va); dfree(&ctx->du);
    dfree(&ctx->st_pos); dfree(&ctx->st_vel); dfree(&ctx->st_half); dfree(&ctx->st_tmp);
    dfree(&ctx->st_tmp1); dfree(&ctx->q_tmp); dfree(&ctx->h_tmp); dfree(&ctx->flags); dfree(&ctx->d_red); dfree(&ctx->d_dt); dfree(&ctx->rho); dfree(&ctx->d_scalars); dfree(&ctx->sm_next);
    dfree(&ctx->box_start); dfree(&ctx->dtb); dfree(&ctx->dtb_next); dfree(&ctx->box_dtmin); dfree(&ctx->box_red);
    dfree(&ctx->box_in); dfree(&ctx->sbox); dfree(&ctx->sbox_tmp); dfree(&ctx->mkey); dfree(&ctx->node_box);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    for (int k = 0; k < 2; k++)
        if (ctx->tune_ev[k]) cudaEventDestroy(ctx->tune_ev[k]);
    if (ctx->tile_order) cudaFree(ctx->tile_order);
    mlp_free(ctx);
    htb_free(ctx);
    rcb_free(ctx);
    graph_free(ctx);
    prof_free(ctx);
    delete ctx;
    return CRK_OK;
}

extern "C" const char *crk_last_error(const crk_ctx *ctx) { return ctx ? ctx->err : "null context"; }

extern "C" int crk_sync(crk_ctx *ctx, void *stream) {
    if (!ctx) return CRK_EINVAL;
    int rc = crk_sync_counters(ctx, (cudaStream_t)stream);
    if (rc) return rc;
    if (ctx->h_counters[CNT_ERR_INPUT])
        return crk_set_error(ctx, CRK_EINVAL, "%llu invalid particle records", ctx->h_counters[CNT_ERR_INPUT]);
    return CRK_OK;
}

// ------------------------------------------------------------------ passes

static int need_built(crk_ctx *ctx) {
    if (!ctx) return CRK_EINVAL;
    if (!ctx->built) return crk_set_error(ctx, CRK_ESTATE, "call crk_build_cells first");
    return CRK_OK;
}

// neighbour lists of the current build (walk 1 + walk 2), built on first need
static int need_lists(crk_ctx *ctx, cudaStream_t s) { return run_lists(ctx, s); }

extern "C" int crk_build_cells(crk_ctx *ctx, int n, const float *pos_h, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n < 0 || (n > 0 && !pos_h)) return crk_set_error(ctx, CRK_EINVAL, "bad n or pos_h");
    if (n > (1 << 30)) return crk_set_error(ctx, CRK_EINVAL, "n beyond 2^30");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->rates_valid = 0;
    int rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s);
    if (rc) return rc;
    rc = finish_build(ctx, s);
    if (rc) {
        ctx->built = 0;
        return rc;
    }
    return CRK_OK;
}

// box of caller row t: the b with box_start[b] <= t < box_start[b+1]
__global__ void k_box_of(int n, int nbox, const int32_t *__restrict__ start, int32_t *__restrict__ box) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    box[t] = lo;
}

int crk::ensure_boxes(crk_ctx *ctx, int n, int nbox) {
    int rc = 0;
    if (nbox > ctx->cap_box) {
        int cap = nbox < 64 ? 64 : nbox;
        rc |= dalloc(ctx, &ctx->box_start, (size_t)cap + 1);
        rc |= dalloc(ctx, &ctx->dtb, (size_t)cap);
        rc |= dalloc(ctx, &ctx->dtb_next, (size_t)cap);
        rc |= dalloc(ctx, &ctx->box_dtmin, (size_t)cap);
        rc |= dalloc(ctx, &ctx->box_red, 8 * (size_t)cap);
        if (rc) return rc;
        ctx->cap_box = cap;
    }
    if (n > ctx->cap_bpart || !ctx->sbox) {
        int cap = n < 4096 ? 4096 : n + n / 8;
        int tiles = (cap + TILE - 1) / TILE;
        rc |= dalloc(ctx, &ctx->box_in, (size_t)cap);
        rc |= dalloc(ctx, &ctx->sbox, (size_t)cap);
        rc |= dalloc(ctx, &ctx->sbox_tmp, (size_t)cap);
        rc |= dalloc(ctx, &ctx->mkey, (size_t)cap);
        rc |= dalloc(ctx, &ctx->node_box, 2 * (size_t)tiles + MAX_LEVELS);
        if (rc) return rc;
        ctx->cap_bpart = cap;
    }
    return CRK_OK;
}

// Validate a host box table and load it; ctx->box_in gets the box of every caller row.
int crk::load_boxes(crk_ctx *ctx, int n, int nbox, const int32_t *box_start, cudaStream_t s) {
    if (nbox < 1 || nbox > 65535 || !box_start) return crk_set_error(ctx, CRK_EINVAL, "bad box table");
    if (box_start[0] != 0 || box_start[nbox] != n)
        return crk_set_error(ctx, CRK_EINVAL, "box table must start at 0 and end at n");
    for (int b = 0; b < nbox; b++)
        if (box_start[b + 1] < box_start[b]) return crk_set_error(ctx, CRK_EINVAL, "box table not ascending");
    int rc = ensure_boxes(ctx, n, nbox);
    if (rc) return rc;
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->box_start, box_start, sizeof(int32_t) * ((size_t)nbox + 1),
                                  cudaMemcpyHostToDevice, s));
    k_box_of<<<grid_for(n, 256), 256, 0, s>>>(n, nbox, ctx->box_start, ctx->box_in);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "box ids");
    CRK_CUDA(ctx, cudaStreamSynchronize(s));   // the host table may be freed after the call
    ctx->nbox = nbox;
    return CRK_OK;
}

extern "C" int crk_build_cells_batched(crk_ctx *ctx, int n, int nbox, const int32_t *box_start,
                                       const float *pos_h, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n < 1 || !pos_h) return crk_set_error(ctx, CRK_EINVAL, "bad n or pos_h");
    if (n > (1 << 30)) return crk_set_error(ctx, CRK_EINVAL, "n beyond 2^30");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->rates_valid = 0;
    int rc = crk_ensure_particles(ctx, n);
    if (!rc) rc = load_boxes(ctx, n, nbox, box_start, s);
    if (!rc) rc = build_cells_sorted(ctx, n, (const float4 *)pos_h, nullptr, s, ctx->box_in);
    if (!rc) rc = finish_build(ctx, s);
    if (rc) {
        ctx->built = 0;
        return rc;
    }
    return CRK_OK;
}

extern "C" int crk_order(crk_ctx *ctx, int32_t *perm, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (!perm) return crk_set_error(ctx, CRK_EINVAL, "null perm");
    if (ctx->n)
        CRK_CUDA(ctx, cudaMemcpyAsync(perm, ctx->perm, 4 * (size_t)ctx->n, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream));
    return CRK_OK;
}

extern "C" int crk_cells(crk_ctx *ctx, uint32_t *keys, int32_t *perm, int32_t *cell_start, int *k_out,
                         void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (ctx->nbox > 1) return crk_set_error(ctx, CRK_ESTATE, "the chaining-mesh table describes one box");
    if (ctx->p.tile_order != 0)
        return crk_set_error(ctx, CRK_ESTATE, "the chaining-mesh table describes the Morton order (tile_order 0)");
    cudaStream_t s = (cudaStream_t)stream;
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    int k = cell_level_host(ctx);
    if (k_out) *k_out = k;
    if (keys && ctx->n) CRK_CUDA(ctx, cudaMemcpyAsync(keys, ctx->keys, 4 * (size_t)ctx->n, cudaMemcpyDeviceToDevice, s));
    if (perm && ctx->n) CRK_CUDA(ctx, cudaMemcpyAsync(perm, ctx->perm, 4 * (size_t)ctx->n, cudaMemcpyDeviceToDevice, s));
    if (cell_start) {
        size_t cnt = ((size_t)1 << (3 * k)) + 1;
        if (ctx->n)
            CRK_CUDA(ctx, cudaMemcpyAsync(cell_start, ctx->cell_start, 4 * cnt, cudaMemcpyDeviceToDevice, s));
        else
            CRK_CUDA(ctx, cudaMemsetAsync(cell_start, 0, 4 * cnt, s));
    }
    CRK_CUDA(ctx, cudaStreamSynchronize(s));
    return CRK_OK;
}

extern "C" int crk_build_stats(crk_ctx *ctx, int *ntiles, long long *g, long long *u, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    rc = crk_sync_counters(ctx, (cudaStream_t)stream);
    if (rc) return rc;
    if (ntiles) *ntiles = ctx->ntiles;
    if (g) *g = ctx->lists_valid ? ctx->entries : 0;
    if (u) *u = (long long)ctx->h_counters[CNT_ULIST];
    return CRK_OK;
}

extern "C" int crk_walk_stats(crk_ctx *ctx, long long *lane_tests, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    rc = crk_sync_counters(ctx, (cudaStream_t)stream);
    if (rc) return rc;
    if (lane_tests) *lane_tests = (long long)ctx->h_counters[CNT_WALK_TESTS];
    return CRK_OK;
}

extern "C" int crk_neighbours(crk_ctx *ctx, int mode, int32_t *count, uint32_t *hash, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if ((ctx->n > 0 && (!count || !hash)) || (mode != 0 && mode != 1))
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    rc = run_neighbours(ctx, mode, ctx->flags, reinterpret_cast<uint32_t *>(ctx->st_tmp1), s);
    if (!rc) rc = scatter_rows(ctx, ctx->flags, count, 1, s);
    if (!rc) rc = scatter_rows(ctx, ctx->st_tmp1, hash, 1, s);
    return rc;
}

extern "C" int crk_neighbour_lists(crk_ctx *ctx, int mode, const long long *offsets, int32_t *lists,
                                   void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if ((ctx->n > 0 && (!offsets || !lists)) || (mode != 0 && mode != 1))
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    if (ctx->volumes_only) return crk_set_error(ctx, CRK_ESTATE, "no neighbour lists in this context");
    return run_export_lists(ctx, mode, offsets, lists, (cudaStream_t)stream);
}

extern "C" int crk_volumes(crk_ctx *ctx, float *V, float *Nngb, long long *pairs, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (!V && ctx->n > 0) return crk_set_error(ctx, CRK_EINVAL, "V is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    rc = run_volumes(ctx, s);
    if (rc) return rc;
    rc = scatter_rows(ctx, ctx->V, V, 1, s);
    if (!rc && Nngb) rc = scatter_rows(ctx, ctx->Nn, Nngb, 1, s);
    if (rc) return rc;
    if (pairs) {
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        *pairs = (long long)ctx->h_counters[CNT_PAIRS_G];
    }
    return CRK_OK;
}

extern "C" int crk_corrections(crk_ctx *ctx, const float *V, const float *vel_u, float *A, float *B,
                               float *gradA, float *gradB, float *gradv, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (ctx->n > 0 && (!V || !A || !B || !gradA || !gradB || (gradv && !vel_u)))
        return crk_set_error(ctx, CRK_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int n = ctx->n;
    rc = need_lists(ctx, s);
    if (rc) return rc;
    rc = gather_rows(ctx, V, ctx->V, 1, s);
    if (!rc && vel_u) rc = gather_rows(ctx, vel_u, ctx->vel, 4, s);
    if (rc) return rc;
    if (n) {
        k_make_qV<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->q4, ctx->V, ctx->qV);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "gather records");
    }
    rc = run_corrections(ctx, gradv != nullptr, s);
    if (rc) return rc;
    if (n) {
        k_unpack_corr<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, ctx->corr, A, B, gradA, gradB);
        ++ctx->launches;
        if (gradv) {
            k_unpack_gv<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, ctx->gv, gradv);
            ++ctx->launches;
        }
        CRK_LAUNCH_CHECK(ctx, "unpack corrections");
    }
    return CRK_OK;
}

static int pack_force_inputs(crk_ctx *ctx, const float *mass, const float *vel_u, const float *V, const float *A,
                             const float *B, const float *gradA, const float *gradB, const float *gradv,
                             cudaStream_t s) {
    int n = ctx->n;
    int rc = need_lists(ctx, s);
    if (!rc) rc = gather_rows(ctx, mass, ctx->mass, 1, s);
    if (!rc) rc = gather_rows(ctx, vel_u, ctx->vel, 4, s);
    if (!rc) rc = gather_rows(ctx, V, ctx->V, 1, s);
    if (rc) return rc;
    if (n) {
        k_pack_corr<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, A, B, gradA, gradB, ctx->corr);
        ++ctx->launches;
        k_pack_gv<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, gradv, ctx->gv);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "pack force inputs");
    }
    return CRK_OK;
}

extern "C" int crk_forces(crk_ctx *ctx, const float *mass, const float *vel_u, const float *V, const float *A,
                          const float *B, const float *gradA, const float *gradB, const float *gradv,
                          float *accel, float *dudt, float *vsig, float *qmax, long long *pairs, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (ctx->n > 0 && (!mass || !vel_u || !V || !A || !B || !gradA || !gradB || !gradv || !accel || !dudt))
        return crk_set_error(ctx, CRK_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    rc = pack_force_inputs(ctx, mass, vel_u, V, A, B, gradA, gradB, gradv, s);
    if (rc) return rc;
    rc = run_forces(ctx, s);
    if (rc) return rc;
    int n = ctx->n;
    if (n) {
        k_unpack_forces<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, ctx->acc, ctx->vq, accel, dudt, vsig, qmax);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "unpack forces");
    }
    if (pairs) {
        rc = crk_sync_counters(ctx, s);
        if (rc) return rc;
        *pairs = (long long)ctx->h_counters[CNT_PAIRS_U];
    }
    return CRK_OK;
}

extern "C" int crk_compatible(crk_ctx *ctx, const float *mass, const float *vel_u, const float *V, const float *A,
                              const float *B, const float *gradA, const float *gradB, const float *gradv,
                              const float *vel_before, const float *vel_after, float *du, void *stream) {
    int rc = need_built(ctx);
    if (rc) return rc;
    if (ctx->n > 0 &&
        (!mass || !vel_u || !V || !A || !B || !gradA || !gradB || !gradv || !vel_before || !vel_after || !du))
        return crk_set_error(ctx, CRK_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    rc = pack_force_inputs(ctx, mass, vel_u, V, A, B, gradA, gradB, gradv, s);
    if (rc) return rc;
    int n = ctx->n;
    if (n) {
        k_pack_v3<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, vel_before, ctx->vb);
        ++ctx->launches;
        k_pack_v3<<<grid_for(n, 256), 256, 0, s>>>(n, ctx->perm, vel_after, ctx->va);
        ++ctx->launches;
        CRK_LAUNCH_CHECK(ctx, "pack kick velocities");
    }
    rc = run_forces(ctx, s);     // F_ij of this evaluation state
    if (!rc) rc = run_compatible(ctx, s);
    if (rc) return rc;
    return scatter_rows(ctx, ctx->du, du, 1, s);
}
