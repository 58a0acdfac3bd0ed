// crk_mlp.cu -- learned smoothing-length proposal.
//
// The paper evolves h with one Thacker update per step (Sec. 2.6, eq:thacker);
// solving eq:hi for each particle is a fixed-point iteration of that update.
// This file proposes the starting point of the iteration with a small network
// and trains the network on converged solutions:
//
//   features  8 per particle from the occupancy of the 27 cells around the
//             particle on a fixed grid of side 2^-kf >= 4 N^(-1/3), the
//             previous h, the compression over the last step dt div v and
//             the previous neighbour count;
//   network   y = s_y (W3 . silu(W2 silu(W1 x + b1) + b2) + b3), 8 -> 64 -> 64 -> 1,
//             s_y = 2^-6 a fixed output scale,
//             BF16 weights and layer inputs, FP32 accumulation and biases, on
//             the tensor cores (mma.sync m16n8k8 for layer 1, m16n8k16 for
//             layer 2, one warp per 16-row tile);
//   proposal  h = h_ref exp(y), h_ref = h_prev (N_res / N_prev)^(1/3) the
//             constant-density solution of eq:hi; h stays h_prev where the previous count
//             already meets the tolerance (the iteration judges and corrects
//             every proposal);
//   training  loss mean (y - log(h_conv / h_ref))^2, forward and backward
//             on the tensor cores, per-block gradient partials summed in a
//             fixed order, Adam on FP32 master weights.
//
// silu(z) = z s(z) with the logistic s(z) = (1 + tanh(z/2)) / 2, evaluated with
// the hardware tanh approximation (one SFU operation per activation).
#include "crk_internal.cuh"

#include <cuda_bf16.h>
#include <math.h>

using namespace crk;

namespace {

constexpr int NP = CRK_MLP_NPARAM;                     // 4801
constexpr int OFF_W1 = 0, OFF_B1 = 512, OFF_W2 = 576, OFF_B2 = 4672, OFF_W3 = 4736, OFF_B3 = 4800;
constexpr int NPART = 4804;                            // per-block partial row: gradient, loss, pad
constexpr int LD = 72;                                 // padded row (bf16) of 64-wide shared tiles
constexpr float Y_SCALE = 0.015625f;                   // fixed output scale s_y = 2^-6

// ------------------------------------------------------------------ small helpers

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ float tanh_sfu(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float logistic(float z) { return fmaf(0.5f, tanh_sfu(0.5f * z), 0.5f); }

// Packed FP32 pairs (one instruction for two IEEE-rounded operations, the
// same results as the scalar ones): the two columns of an mma accumulator
// pair sit in adjacent registers.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(unsigned long long v) {
    float2 f;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
    return f;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// silu of an accumulator pair (z0, z1) = (z0 s(z0), z1 s(z1)); with DS also s(1 + z(1 - s))
template <bool DS>
__device__ __forceinline__ float2 silu2(float z0, float z1, float2 *ds = nullptr) {
    const unsigned long long half = pk2(0.5f, 0.5f);
    const unsigned long long z = pk2(z0, z1);
    const float2 hz = up2(mul2(half, z));
    const unsigned long long th = pk2(tanh_sfu(hz.x), tanh_sfu(hz.y));
    const unsigned long long sg = fma2(half, th, half);
    if (DS) {
        const float2 sv = up2(sg);
        const unsigned long long oms = pk2(1.f - sv.x, 1.f - sv.y);
        *ds = up2(mul2(sg, fma2(z, oms, pk2(1.f, 1.f))));
    }
    return up2(mul2(z, sg));
}

// D += A (16x8, row) B (8x8, col); bf16 in, f32 accumulate
__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// D += A (16x16, row) B (16x8, col); bf16 in, f32 accumulate
__device__ __forceinline__ void mma_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// ------------------------------------------------------------------ features

struct FeatArgs {
    int n;
    int kf;                  // feature grid level
    const float4 *pos_h;     // caller order (x, y, z, h)
    const float *gradv;      // gv_stride n or null (div v = trace: entries 0, 4, 8 of a row)
    int gv_stride;           // 9 (caller's 3x3 rows) or 12 (the engine's padded records)
    const float *Nngb;       // n or null
    const int32_t *fcnt;     // 8^kf cell counts
    float dt;                // step of the state (feature 6 = dt div v)
    float log_cbrt_n;        // log(N^(1/3)) = -log(Delta)
    float inv_N_res;
    float N_res;
};

// h_ref: the constant-density solution of eq:hi from the previous count
// (h (N_res / N)^(1/3)), or h without a count.
__device__ __forceinline__ float h_reference(const FeatArgs &a, float h, float N) {
    return a.Nngb ? h * cbrtf(a.N_res / N) : h;
}

__global__ void k_feat_count(int n, int kf, const float4 *__restrict__ pos_h, int32_t *__restrict__ fcnt,
                             unsigned long long *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    uint32_t cell = 0;
    if (i < n) {
        float4 p = pos_h[i];
        ok = p.x >= 0.f && p.x < 1.f && p.y >= 0.f && p.y < 1.f && p.z >= 0.f && p.z < 1.f && p.w > 0.f &&
             p.w < 1.f;   // NaN fails every comparison
        if (ok) {
            uint32_t sh = 32 - kf;
            uint32_t cx = to_fixed(p.x) >> sh, cy = to_fixed(p.y) >> sh, cz = to_fixed(p.z) >> sh;
            cell = (cz << (2 * kf)) | (cy << kf) | cx;
        } else {
            atomicAdd(err, 1ull);
        }
    }
    // one atomic per distinct cell of the warp
    unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
        unsigned peers = __match_any_sync(act, cell);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&fcnt[cell], __popc(peers));
    }
}

// Features 2t and 2t+1 of row i for lane t (0..3) of a quad; all four lanes of
// the quad must call it for the same row.  Lanes 0..2 each sum one z-plane of
// the 27 cells; the class sums are combined across the quad.
__device__ __forceinline__ float2 quad_features(const FeatArgs &a, int i, int t, float &h_out, float &N_out) {
    bool valid = i < a.n;
    float4 p = valid ? a.pos_h[i] : make_float4(0.5f, 0.5f, 0.5f, 1.f);
    int g = 1 << a.kf;
    uint32_t sh = 32 - a.kf;
    int cx = (int)(to_fixed(p.x) >> sh), cy = (int)(to_fixed(p.y) >> sh), cz = (int)(to_fixed(p.z) >> sh);
    float cls[4] = {0.f, 0.f, 0.f, 0.f};   // own, face, edge, corner
    if (t < 3 && valid) {
        int dz = t - 1;
        int z = (cz + dz + g) & (g - 1);
#pragma unroll
        for (int dy = -1; dy <= 1; dy++) {
            int y = (cy + dy + g) & (g - 1);
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) {
                int x = (cx + dx + g) & (g - 1);
                float c = (float)__ldg(&a.fcnt[((size_t)z << (2 * a.kf)) | ((size_t)y << a.kf) | (size_t)x]);
                int m = (dx != 0) + (dy != 0) + (dz != 0);
                cls[m] += c;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        cls[k] += __shfl_xor_sync(0xffffffffu, cls[k], 1);
        cls[k] += __shfl_xor_sync(0xffffffffu, cls[k], 2);
    }
    float h = p.w;
    float N = (a.Nngb && valid) ? __ldg(&a.Nngb[i]) : 0.f;
    h_out = h;
    N_out = N;
    float2 f = make_float2(0.f, 0.f);
    if (!valid) return f;
    if (t == 0) {
        f.x = __logf(1.f + cls[0]);   // counts are integers: 1 + c is exact
        f.y = __logf(1.f + cls[1]);
    } else if (t == 1) {
        f.x = __logf(1.f + cls[2]);
        f.y = __logf(1.f + cls[3]);
    } else if (t == 2) {
        f.x = __logf(1.f + (cls[0] + cls[1] + cls[2] + cls[3]));
        f.y = __logf(h) + a.log_cbrt_n;
    } else {
        float dv = 0.f;
        if (a.gradv) {
            const float *gv = a.gradv + (size_t)a.gv_stride * i;
            dv = __ldg(gv) + __ldg(gv + 4) + __ldg(gv + 8);
        }
        f.x = a.dt * dv;
        f.y = a.Nngb ? __logf(N * a.inv_N_res) : 0.f;
    }
    return f;
}

// feat[8i..8i+7] and, with pos_conv, target[i] = log(h_conv / h_prev)
__global__ void k_features(FeatArgs a, const float4 *__restrict__ pos_conv, float *__restrict__ feat,
                           float *__restrict__ target) {
    int lane = threadIdx.x & 31;
    int t = lane & 3;
    // every lane of the warp takes part in the quad shuffles; rows >= n only skip the stores
    int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 2);
    float h, N;
    float2 f = quad_features(a, i, t, h, N);
    if (i < a.n) {
        reinterpret_cast<float2 *>(feat)[4 * (size_t)i + t] = f;
        if (t == 0 && pos_conv && target) target[i] = logf(pos_conv[i].w / h_reference(a, h, N));
    }
}

}  // namespace

// ------------------------------------------------------------------ forward

namespace {

// Weights of one block in shared memory: BF16 W1 (64x8) and W2 (64 x LD rows),
// FP32 biases and the BF16-rounded output row W3.
struct FwdShm {
    __nv_bfloat16 w1[64 * 8];
    __nv_bfloat16 w2[64 * LD];
    float b1[64], b2[64], w3[64];
};

__device__ __forceinline__ void stage_fwd(const float *__restrict__ W, FwdShm &S) {
    for (int k = threadIdx.x; k < 512; k += blockDim.x) S.w1[k] = __float2bfloat16_rn(W[OFF_W1 + k]);
    for (int k = threadIdx.x; k < 4096; k += blockDim.x)
        S.w2[(k >> 6) * LD + (k & 63)] = __float2bfloat16_rn(W[OFF_W2 + k]);
    for (int k = threadIdx.x; k < 64; k += blockDim.x) {
        S.b1[k] = W[OFF_B1 + k];
        S.b2[k] = W[OFF_B2 + k];
        S.w3[k] = bf16r(W[OFF_W3 + k]);
    }
}

// Layer 1 of a 16-row tile: z1 = x W1^T + b1 in the mma accumulator layout
// (lane g = lane/4, t = lane%4 holds rows g and g+8, columns 8j+2t and 8j+2t+1
// of n-tile j).  Returns the BF16 activations as the A fragments of layer 2
// (k-step kk covers columns 16kk..16kk+15) and, with DS, silu'(z1).
template <bool DS>
__device__ __forceinline__ void layer1(uint32_t xa0, uint32_t xa1, const uint32_t (&w1f)[8], const FwdShm &S, int t,
                                       uint32_t (&A1)[4][4], float (&ds1)[8][4]) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
        float c0 = S.b1[8 * j + 2 * t], c1 = S.b1[8 * j + 2 * t + 1];
        float d[4] = {c0, c1, c0, c1};
        mma_k8(d, xa0, xa1, w1f[j]);
        float2 g0, g1;
        const float2 a01 = silu2<DS>(d[0], d[1], &g0), a23 = silu2<DS>(d[2], d[3], &g1);
        if (DS) {
            ds1[j][0] = g0.x; ds1[j][1] = g0.y;
            ds1[j][2] = g1.x; ds1[j][3] = g1.y;
        }
        A1[j >> 1][2 * (j & 1) + 0] = pack_bf16(a01.x, a01.y);   // row g
        A1[j >> 1][2 * (j & 1) + 1] = pack_bf16(a23.x, a23.y);   // row g + 8
    }
}

// Layer 2 n-tile j: z2 = a1 W2^T + b2 (B fragment: W2 row 8j+g, k = 16kk+2t).
__device__ __forceinline__ void layer2_tile(int j, const uint32_t (&A1)[4][4], const FwdShm &S, int g, int t,
                                            float (&d)[4]) {
    float c0 = S.b2[8 * j + 2 * t], c1 = S.b2[8 * j + 2 * t + 1];
    d[0] = c0; d[1] = c1; d[2] = c0; d[3] = c1;
    const __nv_bfloat16 *wr = S.w2 + (8 * j + g) * LD + 2 * t;
#pragma unroll
    for (int kk = 0; kk < 4; kk++) mma_k16(d, A1[kk], lds32(wr + 16 * kk), lds32(wr + 16 * kk + 8));
}

__device__ __forceinline__ void load_w1f(const FwdShm &S, int g, int t, uint32_t (&w1f)[8]) {
#pragma unroll
    for (int j = 0; j < 8; j++) w1f[j] = lds32(S.w1 + (8 * j + g) * 8 + 2 * t);
}

__device__ __forceinline__ float quad_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// Inference: MODE 0 reads feat (8n, row-major) and writes y; MODE 1 computes
// the features in place and writes the proposal into pos.w.  One warp per
// 16-row tile, tiles strided over the grid.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_mlp_fwd(int n, const float *__restrict__ W, const float *__restrict__ feat,
                                                  float *__restrict__ y_out, FeatArgs fa, float4 *pos_out, float tol,
                                                  float h_min, float h_max, float N_res) {
    __shared__ __align__(16) FwdShm S;
    stage_fwd(W, S);
    float b3 = W[OFF_B3];
    __syncthreads();
    int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t w1f[8];
    load_w1f(S, g, t, w1f);
    int wpb = blockDim.x >> 5;
    int ntile = (n + 15) >> 4;
    for (int tile = blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntile; tile += gridDim.x * wpb) {
        int r0 = tile * 16 + g, r1 = r0 + 8;
        float2 x0 = make_float2(0.f, 0.f), x1 = x0;
        float h0 = 0.f, h1 = 0.f, N0 = 0.f, N1 = 0.f;
        if (MODE == 0) {
            if (r0 < n) x0 = __ldg(reinterpret_cast<const float2 *>(feat) + 4 * (size_t)r0 + t);
            if (r1 < n) x1 = __ldg(reinterpret_cast<const float2 *>(feat) + 4 * (size_t)r1 + t);
        } else {
            x0 = quad_features(fa, r0, t, h0, N0);
            x1 = quad_features(fa, r1, t, h1, N1);
        }
        uint32_t A1[4][4];
        float unused[8][4];
        layer1<false>(pack_bf16(x0.x, x0.y), pack_bf16(x1.x, x1.y), w1f, S, t, A1, unused);
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float d[4];
            layer2_tile(j, A1, S, g, t, d);
            float wa = S.w3[8 * j + 2 * t], wb = S.w3[8 * j + 2 * t + 1];
            const float2 a01 = silu2<false>(d[0], d[1]), a23 = silu2<false>(d[2], d[3]);
            y0 = fmaf(wa, bf16r(a01.x), fmaf(wb, bf16r(a01.y), y0));
            y1 = fmaf(wa, bf16r(a23.x), fmaf(wb, bf16r(a23.y), y1));
        }
        y0 = Y_SCALE * (quad_sum(y0) + b3);
        y1 = Y_SCALE * (quad_sum(y1) + b3);
        if (t == 0 && MODE == 0) {
            if (r0 < n) y_out[r0] = y0;
            if (r1 < n) y_out[r1] = y1;
        }
        if (t == 0 && MODE == 1) {
#pragma unroll
            for (int e = 0; e < 2; e++) {
                int r = e ? r1 : r0;
                float h = e ? h1 : h0, N = e ? N1 : N0, y = e ? y1 : y0;
                bool done = fa.Nngb && fabsf(cbrtf(N_res / N) - 1.f) <= tol;
                float hn = done ? h : fminf(fmaxf(h_reference(fa, h, N) * expf(y), h_min), h_max);
                if (r < n) pos_out[r].w = hn;
            }
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ training

namespace {

// Shared memory of the gradient kernel: the forward weights, W2^T for the
// backward product, and the transposed BF16 tiles of one 64-row chunk that
// feed the weight-gradient products (rows of the chunk are the k dimension).
struct GradShm {
    FwdShm f;
    __nv_bfloat16 w2t[64 * LD];   // W2^T [in][out]
    __nv_bfloat16 a1t[64 * LD];   // silu(z1)^T [in][row]
    __nv_bfloat16 d2t[64 * LD];   // dL/dz2 ^T [out][row]
    __nv_bfloat16 d1t[64 * LD];   // dL/dz1 ^T [out][row]
    __nv_bfloat16 xt[8 * LD];     // x^T [in][row]
};

struct TrainArgs {
    int n;                        // rows of the data set
    int batch;                    // rows of this step
    long long step;               // < 0: rows 0..batch-1 in order; else sampled
    unsigned long long seed;
    const float *feat, *target, *W;
    const int32_t *rows;          // sampled rows come from rows[0..n_rows) (null: all n)
    int n_rows;
    float two_over_B;
    float *part;                  // [gridDim.x][NPART]
};

// Row r of a sampled batch: SplitMix64 (Steele, Lea, Flood 2014) of a
// per-sample counter, mapped to [0, n) by a 32x32-bit multiply-shift.
__device__ __forceinline__ int sample_row(const TrainArgs &a, int r) {
    if (a.step < 0) return r;
    unsigned long long z = a.seed + ((unsigned long long)a.step * (unsigned long long)a.batch + (unsigned long long)r + 1ull) *
                                        0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if (a.rows) return __ldg(a.rows + (int)(((z >> 32) * (unsigned long long)a.n_rows) >> 32));
    return (int)(((z >> 32) * (unsigned long long)a.n) >> 32);
}

// flag[i] = 1 where the judge hands particle i to the proposal
__global__ void k_select_flags(int n, const float *__restrict__ Nngb, float N_res, float tol,
                               uint32_t *__restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = fabsf(cbrtf(N_res / Nngb[i]) - 1.f) > tol ? 1u : 0u;
}

__global__ void k_select_rows(int n, int base, const uint32_t *__restrict__ flag, const uint32_t *__restrict__ ofs,
                              int32_t *__restrict__ rows, int *count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) rows[ofs[i]] = base + i;
    if (i == n - 1) *count = (int)(ofs[i] + flag[i]);
}

__device__ __forceinline__ float lo_bf16(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float hi_bf16(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void st_bf16(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__global__ void __launch_bounds__(128) k_mlp_grad(TrainArgs a) {
    extern __shared__ __align__(16) unsigned char shm_raw[];
    GradShm &S = *reinterpret_cast<GradShm *>(shm_raw);
    stage_fwd(a.W, S.f);
    for (int k = threadIdx.x; k < 4096; k += blockDim.x)
        S.w2t[(k & 63) * LD + (k >> 6)] = __float2bfloat16_rn(a.W[OFF_W2 + k]);
    float b3 = a.W[OFF_B3];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t w1f[8];
    load_w1f(S.f, g, t, w1f);

    float gw2[8][4], gw1[4], gw3[8][2], gb1[8][2], gb2[8][2], gb3 = 0.f, loss = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
#pragma unroll
        for (int c = 0; c < 4; c++) gw2[j][c] = 0.f;
#pragma unroll
        for (int e = 0; e < 2; e++) gw3[j][e] = gb1[j][e] = gb2[j][e] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) gw1[c] = 0.f;

    const int rr0 = 16 * w + g, rr1 = rr0 + 8;     // rows of this lane within the chunk
    const int nchunk = (a.batch + 63) >> 6;
    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int b0 = ch * 64 + rr0, b1 = ch * 64 + rr1;
        const bool v0 = b0 < a.batch, v1 = b1 < a.batch;
        const int i0 = v0 ? sample_row(a, b0) : 0, i1 = v1 ? sample_row(a, b1) : 0;
        float2 x0 = make_float2(0.f, 0.f), x1 = x0;
        float t0 = 0.f, t1 = 0.f;
        if (v0) {
            x0 = __ldg(reinterpret_cast<const float2 *>(a.feat) + 4 * (size_t)i0 + t);
            t0 = __ldg(a.target + i0);
        }
        if (v1) {
            x1 = __ldg(reinterpret_cast<const float2 *>(a.feat) + 4 * (size_t)i1 + t);
            t1 = __ldg(a.target + i1);
        }
        const uint32_t xa0 = pack_bf16(x0.x, x0.y), xa1 = pack_bf16(x1.x, x1.y);

        // forward, keeping silu' of both layers and the BF16 layer-2 outputs
        uint32_t A1[4][4];
        float ds1[8][4];
        layer1<true>(xa0, xa1, w1f, S.f, t, A1, ds1);
        float a2[8][4], ds2[8][4];
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float d[4];
            layer2_tile(j, A1, S.f, g, t, d);
            float2 g0, g1;
            const float2 a01 = silu2<true>(d[0], d[1], &g0), a23 = silu2<true>(d[2], d[3], &g1);
            a2[j][0] = bf16r(a01.x); a2[j][1] = bf16r(a01.y); a2[j][2] = bf16r(a23.x); a2[j][3] = bf16r(a23.y);
            ds2[j][0] = g0.x; ds2[j][1] = g0.y; ds2[j][2] = g1.x; ds2[j][3] = g1.y;
            float wa = S.f.w3[8 * j + 2 * t], wb = S.f.w3[8 * j + 2 * t + 1];
            y0 = fmaf(wa, a2[j][0], fmaf(wb, a2[j][1], y0));
            y1 = fmaf(wa, a2[j][2], fmaf(wb, a2[j][3], y1));
        }
        y0 = Y_SCALE * (quad_sum(y0) + b3);
        y1 = Y_SCALE * (quad_sum(y1) + b3);
        const float r0 = v0 ? y0 - t0 : 0.f, r1 = v1 ? y1 - t1 : 0.f;
        if (t == 0) {
            loss = fmaf(r0, r0, fmaf(r1, r1, loss));
        }
        const float dy0 = r0 * a.two_over_B, dy1 = r1 * a.two_over_B;
        if (t == 0) gb3 += dy0 + dy1;

        // output layer and dL/dz2
        uint32_t D2[4][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float dz[4];
#pragma unroll
            for (int e = 0; e < 2; e++) {
                gw3[j][e] = fmaf(a2[j][e], dy0, fmaf(a2[j][2 + e], dy1, gw3[j][e]));
                float w3v = S.f.w3[8 * j + 2 * t + e];
                dz[e] = dy0 * w3v * ds2[j][e];
                dz[2 + e] = dy1 * w3v * ds2[j][2 + e];
                gb2[j][e] += dz[e] + dz[2 + e];
            }
            D2[j >> 1][2 * (j & 1) + 0] = pack_bf16(dz[0], dz[1]);
            D2[j >> 1][2 * (j & 1) + 1] = pack_bf16(dz[2], dz[3]);
        }

        // stage transposed x, silu(z1) and dL/dz2 (the BF16 values the products use)
        st_bf16(S.xt + (2 * t) * LD + rr0, x0.x);
        st_bf16(S.xt + (2 * t + 1) * LD + rr0, x0.y);
        st_bf16(S.xt + (2 * t) * LD + rr1, x1.x);
        st_bf16(S.xt + (2 * t + 1) * LD + rr1, x1.y);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int col = 8 * j + 2 * t;
            const uint32_t ar0 = A1[j >> 1][2 * (j & 1)], ar1 = A1[j >> 1][2 * (j & 1) + 1];
            const uint32_t dr0 = D2[j >> 1][2 * (j & 1)], dr1 = D2[j >> 1][2 * (j & 1) + 1];
            st_bf16(S.a1t + col * LD + rr0, lo_bf16(ar0));
            st_bf16(S.a1t + (col + 1) * LD + rr0, hi_bf16(ar0));
            st_bf16(S.a1t + col * LD + rr1, lo_bf16(ar1));
            st_bf16(S.a1t + (col + 1) * LD + rr1, hi_bf16(ar1));
            st_bf16(S.d2t + col * LD + rr0, lo_bf16(dr0));
            st_bf16(S.d2t + (col + 1) * LD + rr0, hi_bf16(dr0));
            st_bf16(S.d2t + col * LD + rr1, lo_bf16(dr1));
            st_bf16(S.d2t + (col + 1) * LD + rr1, hi_bf16(dr1));
        }

        // dL/dz1 = (dL/dz2 W2) * silu'(z1)  (B fragment: W2^T row 8j+g, k = out)
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16 *wr = S.w2t + (8 * j + g) * LD + 2 * t;
#pragma unroll
            for (int kk = 0; kk < 4; kk++) mma_k16(d, D2[kk], lds32(wr + 16 * kk), lds32(wr + 16 * kk + 8));
            const int col = 8 * j + 2 * t;
#pragma unroll
            for (int c = 0; c < 4; c++) d[c] *= ds1[j][c];
            gb1[j][0] += d[0] + d[2];
            gb1[j][1] += d[1] + d[3];
            st_bf16(S.d1t + col * LD + rr0, d[0]);
            st_bf16(S.d1t + (col + 1) * LD + rr0, d[1]);
            st_bf16(S.d1t + col * LD + rr1, d[2]);
            st_bf16(S.d1t + (col + 1) * LD + rr1, d[3]);
        }
        __syncthreads();

        // weight gradients over the chunk's 64 rows: warp w owns outputs 16w..16w+15
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            uint32_t A[4];
            const __nv_bfloat16 *ar = S.d2t + (16 * w + g) * LD + 16 * kk + 2 * t;
            A[0] = lds32(ar);
            A[1] = lds32(ar + 8 * LD);
            A[2] = lds32(ar + 8);
            A[3] = lds32(ar + 8 * LD + 8);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const __nv_bfloat16 *br = S.a1t + (8 * j + g) * LD + 16 * kk + 2 * t;
                mma_k16(gw2[j], A, lds32(br), lds32(br + 8));
            }
            const __nv_bfloat16 *a1r = S.d1t + (16 * w + g) * LD + 16 * kk + 2 * t;
            A[0] = lds32(a1r);
            A[1] = lds32(a1r + 8 * LD);
            A[2] = lds32(a1r + 8);
            A[3] = lds32(a1r + 8 * LD + 8);
            const __nv_bfloat16 *xr = S.xt + g * LD + 16 * kk + 2 * t;
            mma_k16(gw1, A, lds32(xr), lds32(xr + 8));
        }
        __syncthreads();
    }

    // per-block partial gradient, parameter order; loss at NP
    float *P = a.part + (size_t)blockIdx.x * NPART;
#pragma unroll
    for (int j = 0; j < 8; j++) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            int o = 16 * w + g + (c >> 1) * 8, i = 8 * j + 2 * t + (c & 1);
            P[OFF_W2 + o * 64 + i] = gw2[j][c];
        }
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        int o = 16 * w + g + (c >> 1) * 8, i = 2 * t + (c & 1);
        P[OFF_W1 + o * 8 + i] = gw1[c];
    }
    // column sums: over the 8 row groups of the warp, then over the 4 warps
    float *red = reinterpret_cast<float *>(S.a1t);    // [4 warps][3][64] + [4][2]
#pragma unroll
    for (int j = 0; j < 8; j++) {
#pragma unroll
        for (int e = 0; e < 2; e++) {
            float v1 = gb1[j][e], v2 = gb2[j][e], v3 = gw3[j][e];
#pragma unroll
            for (int m = 4; m < 32; m <<= 1) {
                v1 += __shfl_xor_sync(0xffffffffu, v1, m);
                v2 += __shfl_xor_sync(0xffffffffu, v2, m);
                v3 += __shfl_xor_sync(0xffffffffu, v3, m);
            }
            if (g == 0) {
                int col = 8 * j + 2 * t + e;
                red[(w * 3 + 0) * 64 + col] = v1;
                red[(w * 3 + 1) * 64 + col] = v2;
                red[(w * 3 + 2) * 64 + col] = v3;
            }
        }
    }
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        gb3 += __shfl_xor_sync(0xffffffffu, gb3, m);
        loss += __shfl_xor_sync(0xffffffffu, loss, m);
    }
    if (lane == 0) {
        red[4 * 3 * 64 + 2 * w] = gb3;
        red[4 * 3 * 64 + 2 * w + 1] = loss;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * 64; k += blockDim.x) {
        int q = k >> 6, col = k & 63;
        float s = red[q * 64 + col] + red[(3 + q) * 64 + col] + red[(6 + q) * 64 + col] + red[(9 + q) * 64 + col];
        int off = q == 0 ? OFF_B1 : (q == 1 ? OFF_B2 : OFF_W3);
        P[off + col] = s;
    }
    if (threadIdx.x == 0) {
        const float *rs = red + 4 * 3 * 64;
        P[OFF_B3] = rs[0] + rs[2] + rs[4] + rs[6];
        P[NP] = rs[1] + rs[3] + rs[5] + rs[7];
    }
}

struct AdamArgs {
    int nblk;
    const float *part;
    float *W, *m, *v;
    float lr, beta1, beta2, eps, corr1, corr2;   // corr = 1 / (1 - beta^t)
    float inv_B;
    float *grad_out;                             // NP or null
    float *loss_out;                             // 1 or null
};

// Sum of the block partials in block order (deterministic), then one Adam
// update (Kingma & Ba 2015) of each master weight; lr = 0 leaves W unchanged.
__global__ void k_adam(AdamArgs a) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float s = 0.f;
    for (int b = 0; b < a.nblk; b++) s += a.part[(size_t)b * NPART + p];
    if (p == NP) {
        if (a.loss_out) *a.loss_out = s * a.inv_B;
        return;
    }
    if (a.grad_out) a.grad_out[p] = s;
    if (a.lr > 0.f) {
        float m = a.beta1 * a.m[p] + (1.f - a.beta1) * s;
        float v = a.beta2 * a.v[p] + (1.f - a.beta2) * s * s;
        a.m[p] = m;
        a.v[p] = v;
        a.W[p] -= a.lr * (m * a.corr1) / (sqrtf(v * a.corr2) + a.eps);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

constexpr float ADAM_BETA1 = 0.9f, ADAM_BETA2 = 0.999f, ADAM_EPS = 1e-8f;

// largest k in [1, 7] with 64 * 8^k <= n: cell side 2^-k >= 4 N^(-1/3)
int feature_level(int n) {
    int k = 1;
    while (k < 7 && (64ll << (3 * (k + 1))) <= (long long)n) k++;
    return k;
}

int count_cells(crk_ctx *ctx, int n, const float4 *pos, int kf, cudaStream_t s) {
    if (!ctx->fcnt) CRK_CUDA(ctx, cudaMalloc((void **)&ctx->fcnt, sizeof(int32_t) << 21));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->fcnt, 0, sizeof(int32_t) << (3 * kf), s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->counters + CNT_MLP_ERR, 0, sizeof(unsigned long long), s));
    k_feat_count<<<grid_for(n, 256), 256, 0, s>>>(n, kf, pos, ctx->fcnt, ctx->counters + CNT_MLP_ERR);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "feature cell count");
    return CRK_OK;
}

int check_records(crk_ctx *ctx, cudaStream_t s) {
    int rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    unsigned long long bad = ctx->h_counters[CNT_MLP_ERR];
    if (bad) return crk_set_error(ctx, CRK_EINVAL, "%llu particle records outside [0,1)^3 or with h outside (0,1)", bad);
    return CRK_OK;
}

FeatArgs feat_args(const crk_ctx *ctx, int n, const float *pos_h, const float *gradv, const float *Nngb, float dt,
                   int kf) {
    FeatArgs a;
    a.n = n;
    a.dt = dt;
    a.kf = kf;
    a.pos_h = reinterpret_cast<const float4 *>(pos_h);
    a.gradv = gradv;
    a.gv_stride = 9;
    a.Nngb = Nngb;
    a.fcnt = ctx->fcnt;
    a.log_cbrt_n = (float)(log((double)n) / 3.0);
    a.inv_N_res = (float)(1.0 / ctx->p.N_res);
    a.N_res = (float)ctx->p.N_res;
    return a;
}

int need_weights(crk_ctx *ctx) {
    if (!ctx) return CRK_EINVAL;
    if (!ctx->mlp_w) return crk_set_error(ctx, CRK_ESTATE, "call crk_mlp_set_weights first");
    return CRK_OK;
}

int fwd_blocks(const crk_ctx *ctx, int n) {
    int tiles = (n + 15) / 16;
    int b = (tiles + 7) / 8;
    int cap = 4 * (ctx->nsm > 0 ? ctx->nsm : 152);
    return b < 1 ? 1 : (b > cap ? cap : b);
}

int train_launch(crk_ctx *ctx, int n, const float *feat, const float *target, const int32_t *rows, int n_rows,
                 int batch, long long step, float lr, unsigned long long seed, float *grad, float *loss,
                 cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        CRK_CUDA(ctx, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(GradShm)));
        attr_set = true;
    }
    int nchunk = (batch + 63) / 64;
    int cap = 4 * (ctx->nsm > 0 ? ctx->nsm : 152);
    int nblk = nchunk < cap ? nchunk : cap;
    if (nblk > ctx->cap_part) {
        if (ctx->mlp_part) cudaFree(ctx->mlp_part);
        ctx->mlp_part = nullptr;
        ctx->cap_part = 0;
        CRK_CUDA(ctx, cudaMalloc((void **)&ctx->mlp_part, sizeof(float) * NPART * (size_t)cap));
        ctx->cap_part = cap;
    }
    TrainArgs ta;
    ta.n = n;
    ta.batch = batch;
    ta.step = step;
    ta.seed = seed;
    ta.feat = feat;
    ta.target = target;
    ta.rows = rows;
    ta.n_rows = n_rows;
    ta.W = ctx->mlp_w;
    ta.two_over_B = 2.f * Y_SCALE / (float)batch;   // dL/dy times dy/d(output layer)
    ta.part = ctx->mlp_part;
    prof_begin(ctx, PROF_MLP_TRAIN, s);
    k_mlp_grad<<<nblk, 128, sizeof(GradShm), s>>>(ta);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "mlp gradient");
    AdamArgs aa;
    aa.nblk = nblk;
    aa.part = ctx->mlp_part;
    aa.W = ctx->mlp_w;
    aa.m = ctx->mlp_m;
    aa.v = ctx->mlp_v;
    aa.lr = lr;
    aa.beta1 = ADAM_BETA1;
    aa.beta2 = ADAM_BETA2;
    aa.eps = ADAM_EPS;
    if (lr > 0.f) ctx->mlp_t++;
    double tt = (double)(ctx->mlp_t > 0 ? ctx->mlp_t : 1);
    aa.corr1 = (float)(1.0 / (1.0 - pow((double)ADAM_BETA1, tt)));
    aa.corr2 = (float)(1.0 / (1.0 - pow((double)ADAM_BETA2, tt)));
    aa.inv_B = 1.f / (float)batch;
    aa.grad_out = grad;
    aa.loss_out = loss;
    k_adam<<<grid_for(NP + 1, 256), 256, 0, s>>>(aa);
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "mlp adam");
    return CRK_OK;
}

}  // namespace

void crk::mlp_free(crk_ctx *ctx) {
    float **fb[] = {&ctx->mlp_w, &ctx->mlp_m, &ctx->mlp_v, &ctx->mlp_part, &ctx->mlp_hist};
    for (float **p : fb) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    if (ctx->fcnt) cudaFree(ctx->fcnt);
    ctx->fcnt = nullptr;
    if (ctx->sel) cudaFree(ctx->sel);
    ctx->sel = nullptr;
    ctx->cap_sel = 0;
    ctx->cap_part = 0;
    ctx->cap_hist_loss = 0;
}

extern "C" int crk_mlp_set_weights(crk_ctx *ctx, const float *w, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (!w) return crk_set_error(ctx, CRK_EINVAL, "null weights");
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->mlp_w) {
        float **fb[] = {&ctx->mlp_w, &ctx->mlp_m, &ctx->mlp_v};
        for (float **p : fb) {
            cudaError_t e = cudaMalloc((void **)p, sizeof(float) * NP);
            if (e != cudaSuccess) {
                mlp_free(ctx);
                return crk_check_cuda(ctx, e, "cudaMalloc");
            }
        }
    }
    CRK_CUDA(ctx, cudaMemcpyAsync(ctx->mlp_w, w, sizeof(float) * NP, cudaMemcpyDefault, s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->mlp_m, 0, sizeof(float) * NP, s));
    CRK_CUDA(ctx, cudaMemsetAsync(ctx->mlp_v, 0, sizeof(float) * NP, s));
    ctx->mlp_t = 0;
    return CRK_OK;
}

extern "C" int crk_mlp_get_weights(crk_ctx *ctx, float *w, void *stream) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (!w) return crk_set_error(ctx, CRK_EINVAL, "null weights");
    CRK_CUDA(ctx, cudaMemcpyAsync(w, ctx->mlp_w, sizeof(float) * NP, cudaMemcpyDefault, (cudaStream_t)stream));
    return CRK_OK;
}

extern "C" int crk_h_features(crk_ctx *ctx, int n, const float *pos_h, const float *gradv, const float *Nngb,
                              float dt, const float *pos_conv, float *feat, float *target, void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n < 0 || n > (1 << 30)) return crk_set_error(ctx, CRK_EINVAL, "bad n");
    if (n == 0) return CRK_OK;
    if (!pos_h || !feat) return crk_set_error(ctx, CRK_EINVAL, "null pos_h or feat");
    if (!(dt >= 0.f)) return crk_set_error(ctx, CRK_EINVAL, "bad dt");
    if ((pos_conv == nullptr) != (target == nullptr))
        return crk_set_error(ctx, CRK_EINVAL, "pos_conv and target go together");
    cudaStream_t s = (cudaStream_t)stream;
    int kf = feature_level(n);
    int rc = count_cells(ctx, n, reinterpret_cast<const float4 *>(pos_h), kf, s);
    if (rc) return rc;
    FeatArgs fa = feat_args(ctx, n, pos_h, gradv, Nngb, dt, kf);
    k_features<<<grid_for(4ll * n, 256), 256, 0, s>>>(fa, reinterpret_cast<const float4 *>(pos_conv), feat, target);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "features");
    return check_records(ctx, s);
}

extern "C" int crk_mlp_forward(crk_ctx *ctx, int n, const float *feat, float *y, void *stream) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (n < 0) return crk_set_error(ctx, CRK_EINVAL, "bad n");
    if (n == 0) return CRK_OK;
    if (!feat || !y) return crk_set_error(ctx, CRK_EINVAL, "null feat or y");
    cudaStream_t s = (cudaStream_t)stream;
    FeatArgs none{};
    prof_begin(ctx, PROF_MLP_FWD, s);
    k_mlp_fwd<0><<<fwd_blocks(ctx, n), 256, 0, s>>>(n, ctx->mlp_w, feat, y, none, nullptr, 0.f, 0.f, 0.f, 0.f);
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "mlp forward");
    return CRK_OK;
}

extern "C" int crk_h_propose(crk_ctx *ctx, int n, float *pos_h, const float *gradv, const float *Nngb, float dt,
                             float tol, void *stream) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (n < 0 || n > (1 << 30)) return crk_set_error(ctx, CRK_EINVAL, "bad n");
    if (n == 0) return CRK_OK;
    if (!pos_h || !(tol >= 0.f) || !(dt >= 0.f)) return crk_set_error(ctx, CRK_EINVAL, "null pos_h, bad tol or dt");
    cudaStream_t s = (cudaStream_t)stream;
    int kf = feature_level(n);
    prof_begin(ctx, PROF_MLP_FWD, s);
    rc = count_cells(ctx, n, reinterpret_cast<const float4 *>(pos_h), kf, s);
    if (rc) return rc;
    FeatArgs fa = feat_args(ctx, n, pos_h, gradv, Nngb, dt, kf);
    k_mlp_fwd<1><<<fwd_blocks(ctx, n), 256, 0, s>>>(n, ctx->mlp_w, nullptr, nullptr, fa,
                                                     reinterpret_cast<float4 *>(pos_h), tol, (float)ctx->p.h_min,
                                                     (float)ctx->p.h_max, (float)ctx->p.N_res);
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "h proposal");
    return check_records(ctx, s);
}

namespace crk {
// The proposal inside a step (sorted order): pos (x, y, z, h) in place, grad v
// from the engine's padded records, the counts Nn of a P1 at the same
// positions and h, dt the step that led to the state.
int propose_sorted(crk_ctx *ctx, int n, float4 *pos, const GvRec *gv, const float *Nn, float dt, float tol,
                   cudaStream_t s) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (n == 0) return CRK_OK;
    int kf = feature_level(n);
    prof_begin(ctx, PROF_MLP_FWD, s);
    rc = count_cells(ctx, n, pos, kf, s);
    if (rc) return rc;
    FeatArgs fa = feat_args(ctx, n, reinterpret_cast<const float *>(pos), reinterpret_cast<const float *>(gv), Nn,
                            dt, kf);
    fa.gv_stride = 12;
    k_mlp_fwd<1><<<fwd_blocks(ctx, n), 256, 0, s>>>(n, ctx->mlp_w, nullptr, nullptr, fa, pos, tol,
                                                     (float)ctx->p.h_min, (float)ctx->p.h_max, (float)ctx->p.N_res);
    ++ctx->launches;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "h proposal");
    return CRK_OK;
}
}  // namespace crk

extern "C" int crk_mlp_train_step(crk_ctx *ctx, int n, const float *feat, const float *target, float lr, float *grad,
                                  float *loss, void *stream) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (n < 1 || !feat || !target || !(lr >= 0.f)) return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    return train_launch(ctx, n, feat, target, nullptr, 0, n, -1, lr, 0ull, grad, loss, (cudaStream_t)stream);
}

extern "C" int crk_h_select(crk_ctx *ctx, int n, const float *Nngb, float tol, int base, int32_t *rows, int *count,
                            void *stream) {
    if (!ctx) return CRK_EINVAL;
    if (n < 0 || !count || !(tol >= 0.f) || base < 0 || (long long)base + n > (1ll << 31) - 1 ||
        (n > 0 && (!Nngb || !rows)))
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    *count = 0;
    if (n == 0) return CRK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (n > ctx->cap_sel) {
        if (ctx->sel) cudaFree(ctx->sel);
        ctx->sel = nullptr;
        ctx->cap_sel = 0;
        CRK_CUDA(ctx, cudaMalloc((void **)&ctx->sel, sizeof(uint32_t) * 2 * (size_t)n));
        ctx->cap_sel = n;
    }
    uint32_t *flag = ctx->sel, *ofs = ctx->sel + n;
    int rc;
    k_select_flags<<<grid_for(n, 256), 256, 0, s>>>(n, Nngb, (float)ctx->p.N_res, tol, flag);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "select flags");
    rc = scan_u32(ctx, flag, ofs, n, s);
    if (rc) return rc;
    int *d_count = reinterpret_cast<int *>(ctx->counters + CNT_MLP_ERR);
    k_select_rows<<<grid_for(n, 256), 256, 0, s>>>(n, base, flag, ofs, rows, d_count);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "select rows");
    rc = crk_sync_counters(ctx, s);
    if (rc) return rc;
    *count = *reinterpret_cast<int *>(ctx->h_counters + CNT_MLP_ERR);
    return CRK_OK;
}

extern "C" int crk_mlp_train(crk_ctx *ctx, int n, const float *feat, const float *target, const int32_t *rows,
                             int n_rows, int batch, int steps, float lr, unsigned long long seed, float *loss_hist,
                             void *stream) {
    int rc = need_weights(ctx);
    if (rc) return rc;
    if (n < 1 || !feat || !target || batch < 1 || steps < 0 || !(lr > 0.f) || (rows && n_rows < 1))
        return crk_set_error(ctx, CRK_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (steps > ctx->cap_hist_loss) {
        if (ctx->mlp_hist) cudaFree(ctx->mlp_hist);
        ctx->mlp_hist = nullptr;
        ctx->cap_hist_loss = 0;
        CRK_CUDA(ctx, cudaMalloc((void **)&ctx->mlp_hist, sizeof(float) * (size_t)steps));
        ctx->cap_hist_loss = steps;
    }
    for (int k = 0; k < steps; k++) {
        rc = train_launch(ctx, n, feat, target, rows, rows ? n_rows : 0, batch, ctx->mlp_t, lr, seed, nullptr,
                          ctx->mlp_hist + k, s);
        if (rc) return rc;
    }
    if (loss_hist && steps > 0) {
        CRK_CUDA(ctx, cudaMemcpyAsync(loss_hist, ctx->mlp_hist, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, s));
        CRK_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return CRK_OK;
}
