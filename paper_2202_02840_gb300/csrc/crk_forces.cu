// crk_forces.cu -- pair-set passes over {(i,j), i != j : |dq|^2 < max(H_i,H_j)^2},
// walking each particle's neighbour list:
//   P4 momentum and direct energy rates with limited artificial viscosity
//      (CRK-HACC Sec. 1.2 eq:mom, eq:eng, eq:visc, eq:mu, eq:hatvi, eq:phi..eq:phiad)
//   P5 compatible energy (Sec. 1.2 eq:compEng .. eq:fij)
//
// Every ordered pair is evaluated from its i side.  The pair function is
// written so that evaluating (j, i) with the negated separation performs the
// same floating-point operations on swapped operands: F_ji == -F_ij bitwise,
// so the pairwise antisymmetry of eq:mom survives rounding.  P4 stores each
// F_ij at its list entry; P5 (run once per half kick) reuses them.
#include "crk_pass.cuh"

// Divisions of the pair force: the hardware reciprocal-based quotient (two
// instructions, about 2 ulp) instead of the IEEE-rounded one (a dozen and a
// branch).  The same operation is applied to swapped operands for (j, i), so
// F_ji = -F_ij stays bitwise exact.
#define FDIV(a, b) __fdividef((a), (b))

namespace crk {

struct FParams {
    float gm1, gamma;      // gamma - 1, gamma
    float inv_nh;          // 1 / n_h
    float eps2;            // eps^2
    float Cl, Cq;
    float eta_crit, inv_eta_fold;
    // comoving variables (Sec. 1.1): scale factor a, adot = da/dt; all 1 / 0 in a static box
    float half_a2;         // a^2 / 2 (eq:mom)
    float inv_a, inv_a2, inv_a4;
    float adot, adot_a;    // adot, adot / a
};

// Per-particle record of the pair-set passes: 160 bytes, five 32-byte sectors
// (one 256-bit load each).  grad v enters the limiter only through the
// quadratic form x . grad v . x, so its symmetric part is kept (6 numbers).
struct __align__(32) FRec {
    float4 w0;      // qx, qy, qz (fixed-point bits), 1/h
    float4 w1;      // cW = 495/(32 pi h^3), cG = -1155/(4 pi h^5), h_hat = h/n_h, V
    float4 w2;      // P, rho, c_s, A
    float4 w3;      // vx, vy, vz, Bx
    float4 w4;      // By, Bz, gAx, gAy
    float4 w5;      // gAz, gB00, gB01, gB02
    float4 w6;      // gB10, gB11, gB12, gB20
    float4 w7;      // gB21, gB22, S_xx, S_yy
    float4 w8;      // S_zz, S_xy, S_xz, S_yz   (S_ab = dv^a/dx^b + dv^b/dx^a for a != b)
    float4 w9;      // unused (keeps records on 32-byte boundaries)
};

__device__ __forceinline__ uint32_t fq(const FRec &r, int k) {
    return __float_as_uint(k == 0 ? r.w0.x : (k == 1 ? r.w0.y : r.w0.z));
}

struct FSrc {
    const uint4 *q4;
    const float *hs;
    const float *rho;      // RK-corrected density, or null for m / V
    const float *V;
    const float4 *vel;
    const float *mass;
    const CorrRec *corr;
    const GvRec *gv;
};

__device__ __forceinline__ FRec load_frec(int j, const FSrc &src, const FParams &fp) {
    FRec r;
    const uint4 q = src.q4[j];
    const float h = src.hs[j], ih = 1.f / h, ih2 = ih * ih, ih3 = ih2 * ih;
    r.w0 = make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), ih);
    float V = src.V[j];
    float4 v = src.vel[j];
    float rho = src.rho ? src.rho[j] : src.mass[j] / V;
    float P = fp.gm1 * rho * v.w;
    CorrRec c = src.corr[j];
    GvRec g = src.gv[j];
    // grad v [a][b]: g0 = (00 01 02 10), g1 = (11 12 20 21), g2 = (22 ...)
    r.w1 = make_float4(KW * ih3, -KG * ih3 * ih2, h * fp.inv_nh, V);
    r.w2 = make_float4(P, rho, sqrtf(fmaxf(fp.gamma * P / rho, 0.f)), c.c0.x);
    r.w3 = make_float4(v.x, v.y, v.z, c.c0.y);
    r.w4 = make_float4(c.c0.z, c.c0.w, c.c1.x, c.c1.y);
    r.w5 = make_float4(c.c1.z, c.c1.w, c.c2.x, c.c2.y);
    r.w6 = make_float4(c.c2.z, c.c2.w, c.c3.x, c.c3.y);
    r.w7 = make_float4(c.c3.z, c.c3.w, g.g0.x, g.g1.x);
    r.w8 = make_float4(g.g2.x, g.g0.y + g.g0.w, g.g0.z + g.g1.z, g.g1.y + g.g1.w);
    r.w9 = make_float4(0.f, 0.f, 0.f, 0.f);
    return r;
}

// eq:gRK for particle a with separation x (= x_a - x_b), kernel value W and
// radial factor G (grad W = G x).
__device__ __forceinline__ void grad_rk(const FRec &a, const float x[3], float W, float G, float out[3]) {
    const float A = a.w2.w;
    const float B[3] = {a.w3.w, a.w4.x, a.w4.y};
    const float gA[3] = {a.w4.z, a.w4.w, a.w5.x};
    const float gB[9] = {a.w5.y, a.w5.z, a.w5.w, a.w6.x, a.w6.y, a.w6.z, a.w6.w, a.w7.x, a.w7.y};
    float sB = fmaf(B[0], x[0], fmaf(B[1], x[1], fmaf(B[2], x[2], 1.f)));
    float sW = sB * W, AW = A * W, AsG = A * sB * G;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        float gBx = fmaf(gB[g], x[0], fmaf(gB[3 + g], x[1], gB[6 + g] * x[2]));
        out[g] = fmaf(gA[g], sW, fmaf(AW, gBx + B[g], AsG * x[g]));
    }
}

// x . grad v . x from the symmetric part and the products xx = (x^2, y^2, z^2, xy, xz, yz)
__device__ __forceinline__ float gv_quad(const FRec &a, const float xx[6]) {
    return fmaf(a.w7.z, xx[0], fmaf(a.w7.w, xx[1], fmaf(a.w8.x, xx[2],
           fmaf(a.w8.y, xx[3], fmaf(a.w8.z, xx[4], a.w8.w * xx[5])))));
}

__device__ __forceinline__ void kern(const FRec &a, float r, bool in, float &W, float &G) {
    float eta = r * a.w0.w;
    float t = fmaxf(1.f - eta, 0.f);
    float t2 = t * t, t5 = t2 * t2 * t;
    W = in ? a.w1.x * t5 * t * fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f) : 0.f;
    G = in ? a.w1.y * fmaf(5.f, eta, 1.f) * t5 : 0.f;
}

struct PairOut {
    float F[3];    // m_a dp_ab/dt = a^2/2 V_a V_b (P~_a + P~_b)(grad W^R_ba - grad W^R_ab)
    float D[3];    // grad W^R_ba - grad W^R_ab
    float Pt_b;    // P_b + Q_b of this pair
    float Q_a;     // Q_a of this pair
    float Q_b;     // Q_b of this pair
};

// One pair of the pair set seen from particle a; x = x_a - x_b.
__device__ __forceinline__ void pair_force(const FRec &a, const FRec &b, const float x[3], float r2,
                                           float r, bool in_a, bool in_b, const FParams &fp, PairOut &o) {
    float Wa, Ga, Wb, Gb;
    kern(a, r, in_a, Wa, Ga);
    kern(b, r, in_b, Wb, Gb);
    const float xn[3] = {-x[0], -x[1], -x[2]};
    float gRa[3], gRb[3];
    grad_rk(a, x, Wa, Ga, gRa);
    grad_rk(b, xn, Wb, Gb, gRb);
#pragma unroll
    for (int g = 0; g < 3; g++) o.D[g] = gRb[g] - gRa[g];

    // limiter, eq:phi .. eq:phiad (x . grad v_a . x and x . grad v_b . x)
    const float xx[6] = {x[0] * x[0], x[1] * x[1], x[2] * x[2], x[0] * x[1], x[0] * x[2], x[1] * x[2]};
    float qa = gv_quad(a, xx);
    float qb = gv_quad(b, xx);
    float qs = qa + qb;
    float phi = 0.f;
    if (qs != 0.f) {
        float is = FDIV(1.f, qs);
        phi = fminf(fmaxf(4.f * (qa * is) * (qb * is), 0.f), 1.f);
    }
    float eta = fminf(r * a.w0.w, r * b.w0.w);
    if (eta < fp.eta_crit) {
        float e = (eta - fp.eta_crit) * fp.inv_eta_fold;
        phi *= __expf(-e * e);
    }
    // projected proper velocity difference along x, eq:hatvi (the state holds
    // p = a v; the projection acts on the peculiar part only):
    // u_ab . x = (p_a - p_b) . x / a - phi/2 (x . grad v_a . x + x . grad v_b . x) + adot r^2
    float vx = fmaf(a.w3.x - b.w3.x, x[0], fmaf(a.w3.y - b.w3.y, x[1], (a.w3.z - b.w3.z) * x[2]));
    float ux = fmaf(fp.adot, r2, fmaf(-0.5f * phi, qs, vx * fp.inv_a));
    // eq:mu (h^/a), eq:visc
    float hha = a.w1.z, hhb = b.w1.z;
    float uxa = ux * fp.inv_a;
    float mua = fminf(FDIV(hha * uxa, fmaf(hha * hha, fp.eps2, r2)), 0.f);
    float mub = fminf(FDIV(hhb * uxa, fmaf(hhb * hhb, fp.eps2, r2)), 0.f);
    float Qa = a.w2.y * mua * fmaf(fp.Cq, mua, -fp.Cl * a.w2.z);
    float Qb = b.w2.y * mub * fmaf(fp.Cq, mub, -fp.Cl * b.w2.z);
    float Pta = a.w2.x + Qa, Ptb = b.w2.x + Qb;
    float cF = fp.half_a2 * (a.w1.w * b.w1.w) * (Pta + Ptb);
#pragma unroll
    for (int g = 0; g < 3; g++) o.F[g] = cF * o.D[g];
    o.Pt_b = Ptb;
    o.Q_a = Qa;
    o.Q_b = Qb;
}

// Per-particle records of the pair-set passes, packed once per evaluation.
__global__ void k_pack_frec(int n, FSrc src, FParams fp, FRec *__restrict__ out, float *__restrict__ sfun) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    FRec r = load_frec(i, src, fp);
    out[i] = r;
    sfun[i] = r.w2.x / powf(r.w2.y, fp.gamma);       // s = P / rho^gamma (eq:fij)
}

__device__ __forceinline__ FRec ldg_frec(const FRec *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    FRec r;
    ldg_v8(q, r.w0, r.w1);
    ldg_v8(q + 2, r.w2, r.w3);
    ldg_v8(q + 4, r.w4, r.w5);
    ldg_v8(q + 6, r.w6, r.w7);
    ldg_v8(q + 8, r.w8, r.w9);
    return r;
}

// ================================================================= P4 forces

template <bool COMP>
struct P4 {
    static constexpr bool GATHER = false;
    static constexpr int UNROLL = 1;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = true;
    static constexpr bool PREFETCH = true;
    static constexpr bool TMA = true;   // has the TMA-fed variant
    using Rec = FRec;
    struct Params {
        const FRec *frec;
        const float *mass;
        FParams fp;
        float4 *acc;   // (ax, ay, az, dudt)
        float2 *vq;    // (vsig, qmax)
        float4 *Fst;   // (F_ij, j bits) per list entry
    };
    static int launch_tma(crk_ctx *ctx, const ListGeom &g, const Params &prm, cudaStream_t s);
    struct IState {
        FRec me;
        float m;
        Acc<COMP> F[3], du;
        float vsig, qmax;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        if (valid) {
            s.me = p.frec[i];
            s.m = p.mass[i];
        } else {
            s.me = FRec{};
            s.me.w0.w = 1.f;
            s.me.w2.y = 1.f;
            s.m = 1.f;
        }
        s.vsig = 0.f;
        s.qmax = 0.f;
    }
    __device__ static void zero(IState &s) {
        for (int g = 0; g < 3; g++) s.F[g] = Acc<COMP>();
        s.du = Acc<COMP>();
        s.vsig = s.qmax = 0.f;
    }
    __device__ static void merge(IState &s, const IState &o) {
        for (int g = 0; g < 3; g++) merge_acc(s.F[g], o.F[g]);
        merge_acc(s.du, o.du);
        s.vsig = fmaxf(s.vsig, o.vsig);
        s.qmax = fmaxf(s.qmax, o.qmax);
    }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) { return ldg_frec(p.frec + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &r, uint32_t e, size_t pos, bool in_i, const Params &p) {
        const bool in_j = in_i ? (e >> 31) != 0u : true;
        int dx = (int)(fq(s.me, 0) - fq(r, 0)), dy = (int)(fq(s.me, 1) - fq(r, 1)), dz = (int)(fq(s.me, 2) - fq(r, 2));
        Sep d = separation(dx, dy, dz);
        float x[3] = {d.x, d.y, d.z};
        PairOut o;
        pair_force(s.me, r, x, d.r2, d.r, in_i, in_j, p.fp, o);
        p.Fst[pos] = make_float4(o.F[0], o.F[1], o.F[2], __uint_as_float(e & 0x3fffffffu));   // F_ij, j
        float dv[3] = {r.w3.x - s.me.w3.x, r.w3.y - s.me.w3.y, r.w3.z - s.me.w3.z};
#pragma unroll
        for (int g = 0; g < 3; g++) s.F[g].add(o.F[g]);
        float wd = fmaf(dv[0], o.D[0], fmaf(dv[1], o.D[1], dv[2] * o.D[2]));
        s.du.add(0.5f * (s.me.w1.w * r.w1.w) * o.Pt_b * wd);
        // (dx_i/dt - dx_j/dt + (adot/a) x_ij).x_ij with dx/dt = p / a^2
        float vx = fmaf(p.fp.adot_a, d.r2, -fmaf(dv[0], x[0], fmaf(dv[1], x[1], dv[2] * x[2])) * p.fp.inv_a2);
        if (vx < 0.f && d.r > 0.f) s.vsig = fmaxf(s.vsig, FDIV(-vx, d.r));
        s.qmax = fmaxf(s.qmax, o.Q_a);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        float im = 1.f / s.m;
        // dp/dt, and du/dt of eq:eng: 1/(2a^2) V V P~ (dx_j/dt - dx_i/dt).D with dx/dt = p / a^2
        p.acc[i] = make_float4(s.F[0].value() * im, s.F[1].value() * im, s.F[2].value() * im,
                               s.du.value() * im * p.fp.inv_a4);
        p.vq[i] = make_float2(s.vsig, s.qmax);
    }
};

// ================================================================= P4 fed by TMA
//
// The same pass as P4's list loop, with each lane's neighbour record brought
// into shared memory by the tensor-memory accelerator instead of five 256-bit
// gathers through L1: per iteration one lane issues eight tile::gather4 loads
// (four records each) of the next entries of all 32 lanes from L2, into the
// other of two stages, and an mbarrier counts their bytes.  The lanes read
// their record from shared memory when its pair comes up, so no registers
// hold records in flight.  Same entries, same order, same pair function:
// bitwise the results of the other variants.  Every wait on the mbarrier is
// bounded; a wait that runs out sets CNT_TMA_ERR, waits (bounded again) for
// the copies still in flight, and the warp returns.
constexpr int TMA_RF = 36;                     // floats of a record P4 reads (w0 .. w8)
constexpr int TMA_SLOT = 640;                  // bytes per gather4: 4 rows of 144 B, 128-byte slots
constexpr int TMA_STAGE = 8 * TMA_SLOT;        // one record per lane
constexpr uint32_t TMA_TX = 32u * TMA_RF * 4u; // bytes a stage receives
constexpr uint32_t TMA_SPIN = 1u << 16;        // try_wait rounds before a wait is given up
constexpr int TMA_WARPS = 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t rounds) {
    uint32_t ok = 0;
    for (uint32_t it = 0; it < rounds && !ok; it++)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return ok != 0;
}

// rows r0..r3 of the record map (x = 0) into 4 x 144 contiguous bytes at dst
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *map, int4 r, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(map), "r"(0), "r"(r.x), "r"(r.y), "r"(r.z), "r"(r.w), "r"(bar)
        : "memory");
}

template <bool COMP>
__global__ void __launch_bounds__(TMA_WARPS * 32) k_p4_tma(ListGeom g, typename P4<COMP>::Params prm,
                                                          const __grid_constant__ CUtensorMap map,
                                                          unsigned long long *err) {
    __shared__ alignas(128) unsigned char stg[TMA_WARPS][2][TMA_STAGE];
    __shared__ alignas(16) int rows[TMA_WARPS][32];
    __shared__ alignas(8) unsigned long long bar[TMA_WARPS][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * TMA_WARPS + w;
    if (tile >= g.ntiles) return;
    const uint32_t bar0 = smem_u32(&bar[w][0]), stg0 = smem_u32(&stg[w][0][0]);   // stage s: + 8 s, + TMA_STAGE s
    if (lane == 0) {
        mbar_init(bar0);
        mbar_init(bar0 + 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    using P = P4<COMP>;
    const int i = tile * TILE + lane;
    const bool valid = i < g.n;
    typename P::IState st;
    P::init(st, i, valid, prm);
    const uint32_t *col0 = g.ent + (size_t)tile * g.kcap * 32 + lane;
    const size_t fb = (size_t)g.fbase[tile] * 32 + lane;
    const int len = min((int)g.len_u[tile], g.kcap);
    const int mg = valid ? min(g.cnt_g[i], g.kcap) : 0;
    const int my = valid ? min(g.cnt_u[i], g.kcap) : 0;
    auto entry = [&](int k) -> uint32_t {
        const int c = k < mg ? k : g.kcap - 1 - (k - mg);
        return __ldg(col0 + (size_t)c * 32);
    };
    // the records of row j of every lane into stage s (lanes without an entry
    // fetch row 0, so that a stage always receives TMA_TX bytes)
    auto issue = [&](int s, uint32_t j) {
        rows[w][lane] = (int)j;
        __syncwarp();
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stage's last reads come first
            mbar_expect_tx(bar0 + 8 * s, TMA_TX);
#pragma unroll
            for (int q = 0; q < 8; q++)
                tma_gather4(stg0 + s * TMA_STAGE + q * TMA_SLOT, &map,
                            *reinterpret_cast<const int4 *>(&rows[w][4 * q]), bar0 + 8 * s);
        }
        __syncwarp();
    };
    uint32_t e0 = my > 0 ? entry(0) : 0u, e1 = my > 1 ? entry(1) : 0u;
    if (len > 0) issue(0, my > 0 ? (e0 & 0x3fffffffu) : 0u);
    uint32_t ph = 0u;   // bit s: the phase stage s waits for next
    const unsigned char *mine = &stg[w][0][0] + (lane >> 2) * TMA_SLOT + (lane & 3) * (TMA_RF * 4);
    for (int k = 0; k < len; k++) {
        const int s = k & 1;
        const uint32_t e = e0;
        if (k + 1 < len) issue(s ^ 1, k + 1 < my ? (e1 & 0x3fffffffu) : 0u);
        e0 = e1;
        e1 = k + 2 < my ? entry(k + 2) : 0u;
        // one decision for the warp: every lane continues, or every lane leaves
        if (!__all_sync(0xffffffffu, mbar_wait(bar0 + 8 * s, (ph >> s) & 1u, TMA_SPIN))) {
            if (lane == 0) atomicAdd(err, 1ull);
            mbar_wait(bar0 + 8 * s, (ph >> s) & 1u, 4 * TMA_SPIN);
            if (k + 1 < len) mbar_wait(bar0 + 8 * (s ^ 1), (ph >> (s ^ 1)) & 1u, 4 * TMA_SPIN);
            return;
        }
        ph ^= 1u << s;
        if (k < my) {
            const float4 *q = reinterpret_cast<const float4 *>(mine + s * TMA_STAGE);
            FRec r;
            r.w0 = q[0];
            r.w1 = q[1];
            r.w2 = q[2];
            r.w3 = q[3];
            r.w4 = q[4];
            r.w5 = q[5];
            r.w6 = q[6];
            r.w7 = q[7];
            r.w8 = q[8];
            r.w9 = make_float4(0.f, 0.f, 0.f, 0.f);
            P::pair(st, r, e, fb + (size_t)k * 32, k < mg, prm);
        }
        __syncwarp();
    }
    if (valid) P::finish(st, i, prm);
}

// The record map: a 2-D tensor of n rows of TMA_RF floats with a row pitch of
// one record (160 B); a box is one row of TMA_RF floats (gather4 takes four).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int frec_tensor_map(crk_ctx *ctx) {
    if (ctx->frec_map_base == (const void *)ctx->frec && ctx->frec_map_rows == ctx->n) return CRK_OK;
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return crk_set_error(ctx, CRK_ECUDA, "cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)TMA_RF, (cuuint64_t)ctx->n};
    const cuuint64_t strides[1] = {(cuuint64_t)sizeof(FRec)};
    const cuuint32_t box[2] = {(cuuint32_t)TMA_RF, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    CUresult r = encode(&ctx->frec_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ctx->frec, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return crk_set_error(ctx, CRK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    ctx->frec_map_base = ctx->frec;
    ctx->frec_map_rows = ctx->n;
    return CRK_OK;
}

template <bool COMP>
int P4<COMP>::launch_tma(crk_ctx *ctx, const ListGeom &g, const Params &prm, cudaStream_t s) {
    int rc = frec_tensor_map(ctx);
    if (rc) return rc;
    k_p4_tma<COMP><<<grid_for(g.ntiles, TMA_WARPS), TMA_WARPS * 32, 0, s>>>(g, prm, ctx->frec_map,
                                                                          ctx->counters + CNT_TMA_ERR);
    return CRK_OK;
}

// ================================================================= P5 compatible energy

// sig = (v + v') of the kick and the entropy s of the evaluation state.
// DUAL: two kicks with the same pair forces in one pass over the stored
// forces (a step's closing kick and the next step's opening kick): sig and
// sig2, du and du2, each sum in the same order as a single pass would take.
// skip (may be null): a device flag set when the sums of this pass were
// already formed by the previous step's dual pass; the pass then reads
// nothing (the caller takes those sums).
// The partition of eq:fij for one pair: f = min(s_i, s_j)/(s_i + s_j) when
// the pair's work and s_i - s_j have the same sign, else max/(s_i + s_j)
// (1/2 when both vanish).  It depends on the pair's entropies only, so the
// two-kick pass forms it once for both kicks.
struct Part {
    float fmn, fmx;
    bool ige;   // s_i >= s_j
};

__device__ __forceinline__ Part partition(float si, float sj) {
    Part p;
    p.ige = si >= sj;
    const float ss = si + sj;
    if (ss != 0.f) {
        const float r = __fdividef(1.f, ss);
        p.fmn = fminf(si, sj) * r;
        p.fmx = fmaxf(si, sj) * r;
    } else {
        p.fmn = p.fmx = 0.5f;
    }
    return p;
}

// 2 Delta E_ij = (v_j + v'_j - v_i - v'_i) . F_ij  (reading of eq:Eij); this
// returns f 2 Delta E_ij, the factor 1/2 being applied to the finished sum
// (an exact scaling)
__device__ __forceinline__ float compat_term(const float4 me, const float4 r, const float4 F, const Part &p) {
    float w = fmaf(r.x - me.x, F.x, fmaf(r.y - me.y, F.y, (r.z - me.z) * F.z));
    return (((w >= 0.f) == p.ige) ? p.fmn : p.fmx) * w;
}

template <bool COMP, bool DUAL = false>
struct P5 {
    static constexpr bool GATHER = false;
    static constexpr int UNROLL = 3;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    static constexpr bool SKIPPABLE = true;
    struct Rec {
        float4 sig, sig2, F;
    };
    struct Params {
        const float4 *sig;    // one kick: sig per particle; two kicks: (sig, sig2) side by side
        const float4 *Fst;
        const float *mass;
        float *du;
        float inv_a4;
        const unsigned long long *skip;
        float *du2;
    };
    struct IState {
        float4 me, me2;
        float m;
        Acc<COMP> du, du2;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        s.me = valid ? p.sig[DUAL ? 2 * (size_t)i : (size_t)i] : z;
        if (DUAL) s.me2 = valid ? p.sig[2 * (size_t)i + 1] : z;
        s.m = valid ? p.mass[i] : 1.f;
    }
    __device__ static void zero(IState &s) {
        s.du = Acc<COMP>();
        s.du2 = Acc<COMP>();
    }
    __device__ static void merge(IState &s, const IState &o) {
        merge_acc(s.du, o.du);
        if (DUAL) merge_acc(s.du2, o.du2);
    }
    // the stored entry carries j (written by P4): the list itself is not read,
    // and the stored (F_ij, j) are what streams from HBM (read ahead)
    static constexpr bool ENTRIES = false;
    using Stored = float4;
    __device__ static Stored stored(size_t pos, const Params &p) { return __ldg(p.Fst + pos); }
    __device__ static Rec load(const float4 &F, size_t, const Params &p) {
        const uint32_t j = __float_as_uint(F.w);
        Rec r;
        if (DUAL)
            ldg_v8(p.sig + 2 * (size_t)j, r.sig, r.sig2);   // both kicks' sums in one 256-bit load
        else
            r.sig = __ldg(p.sig + j);
        r.F = F;
        return r;
    }
    __device__ static void pair(IState &s, const Rec &rec, const float4 &, size_t, bool, const Params &) {
        const Part pt = partition(s.me.w, rec.sig.w);   // both kicks: s of the evaluation state
        s.du.add(compat_term(s.me, rec.sig, rec.F, pt));
        if (DUAL) s.du2.add(compat_term(s.me2, rec.sig2, rec.F, pt));
    }
    // eq:compEng2: 1/(2 a^4) (p_j + p'_j - p_i - p'_i) . dp_ij/dt
    __device__ static void finish(IState &s, int i, const Params &p) {
        p.du[i] = 0.5f * s.du.value() / s.m * p.inv_a4;
        if (DUAL) p.du2[i] = 0.5f * s.du2.value() / s.m * p.inv_a4;
    }
};

// ================================================================= pair-once form
//
// Each unordered pair of the pair set is evaluated once, by its owner: the
// particle with the lower sorted index.  Lane i of tile I takes the entries
// of its list with j > i, which are a suffix of its gather entries and a
// suffix of its other entries (the walk records where they start), merged in
// increasing j: lane i then meets the candidate tiles of I in increasing
// order, the order of I's tile list.  j's share of a pair (-F_ij and the
// terms of j's other sums) goes to a ring of PO_W rows of 32 slots in shared
// memory (row: candidate tile mod PO_W, slot: j's lane).  Lanes that hit one
// slot in the same step add in lane order (match_any), so the sums repeat
// bitwise.  A lane more than PO_W - 1 candidate tiles ahead of the slowest
// lane waits.  When every lane has passed a candidate tile J, its ring row is
// written to J's row of j-side sums for the tile pair: the entry (J, I) of
// J's tile list (po_rev).  A last pass adds, for each particle j, the rows of
// the candidate tiles K <= J of J's tile list, in list order, to j's own
// sums.  The tile lists are symmetric (the tile-pair test is), so every pair
// (I, J) with I <= J has its row, and every row with K <= J is written once.

constexpr int PO_W = 8;        // candidate tiles the ring spans
constexpr int PO_WARPS = 4;    // tiles per CTA
constexpr int PO_CMAX = 128;   // candidate tiles (from the tile's own on) staged in shared memory
constexpr uint32_t PO_NONE = 0xffffffffu;

struct POGeom {
    int n, ntiles, kcap;
    const uint32_t *fbase;        // per-tile stored-force base, units of 32 entries
    const int32_t *cnt_g, *cnt_u;
    const int2 *lowc;             // per particle: gather and other entries with j < i
    const uint32_t *ent;
    const uint2 *tofs;            // pair-set tile lists: (offset, count) per tile
    const uint32_t *tlist;
    const uint32_t *rev;          // entry (I, J), J >= I -> entry (J, I); PO_NONE if missing
    const int32_t *self;          // position of each tile in its own list (-1 if missing)
};

// Reverse index of the tile lists (each list ascending): for entry (I, J)
// with J > I the position of I in J's list, by bisection; J == I gives the
// tile's own position.  A missing reverse (which the symmetric tile-pair
// test rules out) is counted in *miss and its row is never written.  The
// lists are copied beside it (copy_ofs, copy_list): the pair-once passes read
// the copy, which stays the lists of this evaluation when the lists are
// refitted before a later kick.
__global__ void k_po_rev(int ntiles, const uint2 *__restrict__ tofs, const uint32_t *__restrict__ tlist,
                         uint32_t *__restrict__ rev, int32_t *__restrict__ self, uint2 *__restrict__ copy_ofs,
                         uint32_t *__restrict__ copy_list, unsigned long long *miss) {
    const int lane = threadIdx.x & 31;
    const int I = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (I >= ntiles) return;
    const uint2 to = tofs[I];
    if (lane == 0) copy_ofs[I] = to;
    bool found = false;
    for (uint32_t c = lane; c < to.y; c += 32) {
        const uint32_t J = tlist[to.x + c];
        copy_list[to.x + c] = J;
        if (J == (uint32_t)I) {
            self[I] = (int32_t)c;
            rev[to.x + c] = to.x + c;
            found = true;
        } else if (J > (uint32_t)I) {
            const uint2 tj = tofs[J];
            uint32_t lo = 0, hi = tj.y;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (tlist[tj.x + mid] < (uint32_t)I) lo = mid + 1; else hi = mid;
            }
            const bool ok = lo < tj.y && tlist[tj.x + lo] == (uint32_t)I;
            rev[to.x + c] = ok ? tj.x + lo : PO_NONE;
            if (!ok) atomicAdd(miss, 1ull);
        }
    }
    if (__ballot_sync(0xffffffffu, found) == 0u && lane == 0) {
        self[I] = -1;
        atomicAdd(miss, 1ull);
    }
}

// Write ring row c (candidate c of this tile's list) to its tile pair's row
// `row` and clear it; lane l takes slot l.
template <class P>
__device__ __forceinline__ void po_flush(const typename P::Params &prm, float (*ring)[P::NS], uint32_t row, int c,
                                         int lane) {
    float *slot = ring[(c % PO_W) * 32 + lane];
    if (row != PO_NONE) P::flush(row, lane, slot, prm);
#pragma unroll
    for (int q = 0; q < P::NS; q++) slot[q] = 0.f;
}

// One tile of a pair-once pass.  P provides NS (floats of a share), Ent (what
// a lane reads per list entry), Rec (the neighbour data), IState and
//   init(IState&, int i, bool valid, const Params&)
//   fetch(const uint32_t *col0, size_t fb, int mg, int kcap, int k, const Params&) -> Ent   (entry k)
//   jof(const Ent&) -> j
//   load(const Ent&, const Params&) -> Rec
//   pair(IState&, const Rec&, const Ent&, size_t pos, bool in_i, const Params&, float share[NS])
//   add(float *slot, const float share[NS]), flush(uint32_t row, int lane, const float *slot, const Params&)
//   finish(IState&, int i, const Params&)          (valid lanes: i's own sums)
template <class P>
__device__ __forceinline__ void po_tile(const POGeom &g, const typename P::Params &prm, int tile, int lane,
                                        float (*ring)[P::NS], uint32_t *stl, uint32_t *srv) {
    using Ent = typename P::Ent;
    const int i = tile * TILE + lane;
    const bool valid = i < g.n;
    typename P::IState st;
    P::init(st, i, valid, prm);
    const uint2 to = g.tofs[tile];
    const int C = (int)to.y;
    const int cself = g.self[tile];
    if (cself < 0) return;   // counted by the reverse index
    // the candidate tiles from this tile on, and their reverse entries
    const int nst = min(C - cself, PO_CMAX);
    for (int q = lane; q < nst; q += 32) {
        stl[q] = __ldg(g.tlist + to.x + cself + q);
        srv[q] = __ldg(g.rev + to.x + cself + q);
    }
    __syncwarp();
    auto tl_at = [&](int c) -> uint32_t {
        return c - cself < PO_CMAX ? stl[c - cself] : __ldg(g.tlist + to.x + c);
    };
    auto rv_at = [&](int c) -> uint32_t { return c - cself < PO_CMAX ? srv[c - cself] : __ldg(g.rev + to.x + c); };
    const uint32_t *col0 = g.ent + (size_t)tile * g.kcap * 32 + lane;
    const size_t fb = (size_t)g.fbase[tile] * 32 + lane;
    const int mg = valid ? min(g.cnt_g[i], g.kcap) : 0;
    const int mu = valid ? min(g.cnt_u[i], g.kcap) : 0;
    const int2 lw = valid ? g.lowc[i] : make_int2(0, 0);
    // owned entries: gather [kg, mg), other [ko, mu) (virtual indices)
    int kg = min(lw.x, mg), ko = mg + min(lw.y, mu - mg);
    Ent eg{}, eo{};
    if (kg < mg) eg = P::fetch(col0, fb, mg, g.kcap, kg, prm);
    if (ko < mu) eo = P::fetch(col0, fb, mg, g.kcap, ko, prm);
    // next owned entry in increasing j (a j is in one of the two segments only)
    auto pick = [&](int &k, Ent &e, bool &gath) -> bool {
        const uint32_t jg = kg < mg ? P::jof(eg) : PO_NONE;
        const uint32_t jo = ko < mu ? P::jof(eo) : PO_NONE;
        if (jg == PO_NONE && jo == PO_NONE) return false;
        if (jg < jo) {
            k = kg; e = eg; gath = true;
            if (++kg < mg) eg = P::fetch(col0, fb, mg, g.kcap, kg, prm);
        } else {
            k = ko; e = eo; gath = false;
            if (++ko < mu) eo = P::fetch(col0, fb, mg, g.kcap, ko, prm);
        }
        return true;
    };
    // position of j's tile in this tile's list (monotone over a lane's entries)
    int cp = cself;
    uint32_t cJ = (uint32_t)tile;
    auto cand = [&](uint32_t j) -> int {
        const uint32_t J = j / TILE;
        while (cJ < J && cp + 1 < C) cJ = tl_at(++cp);
        return cp;
    };
    int k = 0;
    Ent e{};
    bool gath = false;
    bool have = pick(k, e, gath);
    typename P::Rec rc{};
    int c = C;
    if (have) {
        rc = P::load(e, prm);
        c = cand(P::jof(e));
    }
    int cf = cself;   // ring rows below cf are written out
    for (;;) {
        const int cm = (int)__reduce_min_sync(0xffffffffu, (unsigned)(have ? c : C));
        if (cf < cm) {
            __syncwarp();
            for (; cf < cm; cf++) po_flush<P>(prm, ring, rv_at(cf), cf, lane);
            __syncwarp();
        }
        if (cm >= C) break;
        const bool go = have && c < cf + PO_W;
        int k2 = 0;
        Ent e2{};
        bool g2 = false, have2 = false;
        typename P::Rec rn{};
        if (go) {
            have2 = pick(k2, e2, g2);
            if (have2) rn = P::load(e2, prm);
        }
        float sh[P::NS];
        if (go) P::pair(st, rc, e, fb + (size_t)k * 32, gath, prm, sh);
        // j's share into the ring: lanes with the same slot add in lane order
        const uint32_t key = ((uint32_t)(c % PO_W) << 5) | (P::jof(e) & 31u);
        unsigned pend = __ballot_sync(0xffffffffu, go);
        while (pend) {
            const bool mine = (pend >> lane) & 1u;
            const unsigned grp = __match_any_sync(0xffffffffu, mine ? key : (0x10000u | (uint32_t)lane));
            const bool lead = mine && (__ffs(grp) - 1 == lane);
            if (lead) P::add(ring[key], sh);
            pend &= ~__ballot_sync(0xffffffffu, lead);
        }
        if (go) {
            have = have2;
            k = k2;
            e = e2;
            gath = g2;
            rc = rn;
            c = have ? cand(P::jof(e)) : C;
        }
    }
    if (valid) P::finish(st, i, prm);
}

template <class P>
__global__ void __launch_bounds__(PO_WARPS * 32) k_po(POGeom g, typename P::Params prm) {
    __shared__ float ring[PO_WARPS][PO_W * 32][P::NS];
    __shared__ uint32_t stl[PO_WARPS][PO_CMAX], srv[PO_WARPS][PO_CMAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * PO_WARPS + w;
    if (tile >= g.ntiles) return;
    if (pass_skipped<P>(prm)) return;
    for (int q = lane; q < PO_W * 32; q += 32)
#pragma unroll
        for (int v = 0; v < P::NS; v++) ring[w][q][v] = 0.f;
    __syncwarp();
    po_tile<P>(g, prm, tile, lane, ring[w], stl[w], srv[w]);
}

// P4 in the pair-once form: the same pair function; i's sums as in P4, and
// j's share -F_ij, 1/2 V_j V_i P~_i (dx_i/dt - dx_j/dt).(grad W^R_ij - grad W^R_ji),
// Q_j of the pair and the pair's signal velocity, each bitwise the term the
// directed form evaluates from j's side.
template <bool COMP>
struct P4PO {
    static constexpr int NS = 6;   // F (3), du, Q, vsig
    using Ent = uint32_t;
    using Rec = FRec;
    using IState = typename P4<COMP>::IState;
    struct Params {
        const FRec *frec;
        const float *mass;
        FParams fp;
        float4 *acc;     // own sums (F, du) here; the row pass completes them
        float2 *vq;
        float4 *Fst;     // (F_ij, j) at the owner's entry
        float4 *rowA;    // (F, du) per (tile-list entry, lane)
        float2 *rowB;    // (Q, vsig)
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        typename P4<COMP>::Params q{p.frec, p.mass, p.fp, p.acc, p.vq, p.Fst};
        P4<COMP>::init(s, i, valid, q);
    }
    __device__ static Ent fetch(const uint32_t *col0, size_t, int mg, int kcap, int k, const Params &) {
        const int c = k < mg ? k : kcap - 1 - (k - mg);
        return __ldg(col0 + (size_t)c * 32);
    }
    __device__ static uint32_t jof(const Ent &e) { return e & 0x3fffffffu; }
    __device__ static Rec load(const Ent &e, const Params &p) { return ldg_frec(p.frec + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &r, const Ent &e, size_t pos, bool in_i, const Params &p,
                                float sh[NS]) {
        const bool in_j = in_i ? (e >> 31) != 0u : true;
        int dx = (int)(fq(s.me, 0) - fq(r, 0)), dy = (int)(fq(s.me, 1) - fq(r, 1)), dz = (int)(fq(s.me, 2) - fq(r, 2));
        Sep d = separation(dx, dy, dz);
        float x[3] = {d.x, d.y, d.z};
        PairOut o;
        pair_force(s.me, r, x, d.r2, d.r, in_i, in_j, p.fp, o);
        p.Fst[pos] = make_float4(o.F[0], o.F[1], o.F[2], __uint_as_float(e & 0x3fffffffu));   // F_ij, j
        float dv[3] = {r.w3.x - s.me.w3.x, r.w3.y - s.me.w3.y, r.w3.z - s.me.w3.z};
#pragma unroll
        for (int g = 0; g < 3; g++) s.F[g].add(o.F[g]);
        float wd = fmaf(dv[0], o.D[0], fmaf(dv[1], o.D[1], dv[2] * o.D[2]));
        const float hvv = 0.5f * (s.me.w1.w * r.w1.w);
        s.du.add(hvv * o.Pt_b * wd);
        float vx = fmaf(p.fp.adot_a, d.r2, -fmaf(dv[0], x[0], fmaf(dv[1], x[1], dv[2] * x[2])) * p.fp.inv_a2);
        const float vs = (vx < 0.f && d.r > 0.f) ? FDIV(-vx, d.r) : 0.f;
        s.vsig = fmaxf(s.vsig, vs);
        s.qmax = fmaxf(s.qmax, o.Q_a);
        sh[0] = -o.F[0];
        sh[1] = -o.F[1];
        sh[2] = -o.F[2];
        sh[3] = hvv * (s.me.w2.x + o.Q_a) * wd;
        sh[4] = o.Q_b;
        sh[5] = vs;
    }
    __device__ static void add(float *slot, const float sh[NS]) {
        slot[0] += sh[0];
        slot[1] += sh[1];
        slot[2] += sh[2];
        slot[3] += sh[3];
        slot[4] = fmaxf(slot[4], sh[4]);
        slot[5] = fmaxf(slot[5], sh[5]);
    }
    __device__ static void flush(uint32_t row, int lane, const float *slot, const Params &p) {
        p.rowA[(size_t)row * 32 + lane] = make_float4(slot[0], slot[1], slot[2], slot[3]);
        p.rowB[(size_t)row * 32 + lane] = make_float2(slot[4], slot[5]);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        p.acc[i] = make_float4(s.F[0].value(), s.F[1].value(), s.F[2].value(), s.du.value());
        p.vq[i] = make_float2(s.vsig, s.qmax);
    }
};

// P4 rows: j's own sums plus the rows of the candidate tiles K <= J of its
// list, in list order; then the scalings of P4's finish.
template <bool COMP>
__global__ void k_p4po_rows(int n, const uint2 *__restrict__ tofs, const int32_t *__restrict__ self,
                            const float4 *__restrict__ rowA, const float2 *__restrict__ rowB,
                            const float *__restrict__ mass, FParams fp, float4 *__restrict__ acc,
                            float2 *__restrict__ vq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int tile = i / TILE, lane = i % TILE;
    const float4 own = acc[i];
    float2 v = vq[i];
    Acc<COMP> F[3], du;
    F[0].add(own.x);
    F[1].add(own.y);
    F[2].add(own.z);
    du.add(own.w);
    const uint32_t x = tofs[tile].x;
    const int cs = self[tile];
    for (int c = 0; c <= cs; c++) {
        const size_t r = ((size_t)x + c) * 32 + lane;
        const float4 a = rowA[r];
        const float2 b = rowB[r];
        F[0].add(a.x);
        F[1].add(a.y);
        F[2].add(a.z);
        du.add(a.w);
        v.x = fmaxf(v.x, b.y);
        v.y = fmaxf(v.y, b.x);
    }
    const float im = 1.f / mass[i];
    acc[i] = make_float4(F[0].value() * im, F[1].value() * im, F[2].value() * im, du.value() * im * fp.inv_a4);
    vq[i] = v;
}

// P5 in the pair-once form over the owner's stored (F_ij, j): i's term as in
// P5 and j's, f_ji 2 Delta E_ji with 2 Delta E_ji = 2 Delta E_ij bitwise and
// the partition of eq:fij taken from j's side.
template <bool COMP, bool DUAL>
struct P5PO {
    static constexpr int NS = 2;   // du (this kick), du2 (the second kick)
    static constexpr bool SKIPPABLE = true;
    using Ent = float4;
    struct Rec {
        float4 sig, sig2;
    };
    using IState = typename P5<COMP, DUAL>::IState;
    struct Params {
        const float4 *sig;
        const float4 *Fst;
        const float *mass;
        float *du;       // own sums here; the row pass completes them
        float inv_a4;
        const unsigned long long *skip;
        float *du2;
        float2 *rowB;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        typename P5<COMP, DUAL>::Params q{p.sig, p.Fst, p.mass, p.du, p.inv_a4, p.skip, p.du2};
        P5<COMP, DUAL>::init(s, i, valid, q);
    }
    __device__ static Ent fetch(const uint32_t *, size_t fb, int, int, int k, const Params &p) {
        return __ldg(p.Fst + fb + (size_t)k * 32);
    }
    __device__ static uint32_t jof(const Ent &F) { return __float_as_uint(F.w); }
    __device__ static Rec load(const Ent &F, const Params &p) {
        const uint32_t j = __float_as_uint(F.w);
        Rec r;
        if (DUAL)
            ldg_v8(p.sig + 2 * (size_t)j, r.sig, r.sig2);
        else
            r.sig = __ldg(p.sig + j);
        return r;
    }
    __device__ static float dotw(const float4 &me, const float4 &r, const float4 &F) {
        return fmaf(r.x - me.x, F.x, fmaf(r.y - me.y, F.y, (r.z - me.z) * F.z));
    }
    __device__ static void pair(IState &s, const Rec &rec, const Ent &F, size_t, bool, const Params &,
                                float sh[NS]) {
        const Part pt = partition(s.me.w, rec.sig.w);
        const bool jge = rec.sig.w >= s.me.w;   // s_j >= s_i: the partition seen from j
        const float w = dotw(s.me, rec.sig, F);
        s.du.add((((w >= 0.f) == pt.ige) ? pt.fmn : pt.fmx) * w);
        sh[0] = (((w >= 0.f) == jge) ? pt.fmn : pt.fmx) * w;
        sh[1] = 0.f;
        if (DUAL) {
            const float w2 = dotw(s.me2, rec.sig2, F);
            s.du2.add((((w2 >= 0.f) == pt.ige) ? pt.fmn : pt.fmx) * w2);
            sh[1] = (((w2 >= 0.f) == jge) ? pt.fmn : pt.fmx) * w2;
        }
    }
    __device__ static void add(float *slot, const float sh[NS]) {
        slot[0] += sh[0];
        slot[1] += sh[1];
    }
    __device__ static void flush(uint32_t row, int lane, const float *slot, const Params &p) {
        p.rowB[(size_t)row * 32 + lane] = make_float2(slot[0], slot[1]);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        p.du[i] = s.du.value();
        if (DUAL) p.du2[i] = s.du2.value();
    }
};

template <bool COMP, bool DUAL>
__global__ void k_p5po_rows(int n, const uint2 *__restrict__ tofs, const int32_t *__restrict__ self,
                            const float2 *__restrict__ rowB, const float *__restrict__ mass, float inv_a4,
                            const unsigned long long *skip, float *__restrict__ du, float *__restrict__ du2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (skip && *(volatile const unsigned long long *)skip) return;
    const int tile = i / TILE, lane = i % TILE;
    Acc<COMP> s1, s2;
    s1.add(du[i]);
    if (DUAL) s2.add(du2[i]);
    const uint32_t x = tofs[tile].x;
    const int cs = self[tile];
    for (int c = 0; c <= cs; c++) {
        const float2 b = rowB[((size_t)x + c) * 32 + lane];
        s1.add(b.x);
        if (DUAL) s2.add(b.y);
    }
    const float m = mass[i];
    du[i] = 0.5f * s1.value() / m * inv_a4;
    if (DUAL) du2[i] = 0.5f * s2.value() / m * inv_a4;
}

static POGeom po_geom(const crk_ctx *ctx) {
    return POGeom{ctx->n,   ctx->ntiles,  ctx->kcap,     ctx->tbase,  ctx->cnt_g,  ctx->cnt_u, ctx->lowc,
                  ctx->ent, ctx->po_tofs, ctx->po_tlist, ctx->po_rev, ctx->po_self};
}

static FParams fparams(const crk_params &c) {
    FParams f;
    f.gamma = (float)c.gamma;
    f.gm1 = (float)(c.gamma - 1.0);
    f.inv_nh = (float)(1.0 / c.n_h);
    f.eps2 = (float)(c.eps * c.eps);
    f.Cl = (float)c.C_l;
    f.Cq = (float)c.C_q;
    f.eta_crit = (float)c.eta_crit;
    f.inv_eta_fold = (float)(1.0 / c.eta_fold);
    f.half_a2 = (float)(0.5 * c.a * c.a);
    f.inv_a = (float)(1.0 / c.a);
    f.inv_a2 = (float)(1.0 / (c.a * c.a));
    f.inv_a4 = (float)(1.0 / (c.a * c.a * c.a * c.a));
    f.adot = (float)c.adot;
    f.adot_a = (float)(c.adot / c.a);
    return f;
}

// kick velocities (w unused) -> sig = (vb + va, s)
__global__ void k_sig(int n, const float4 *__restrict__ vb, const float4 *__restrict__ va,
                      const float *__restrict__ sfun, float4 *__restrict__ sig) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 b = vb[i], a = va[i];
    sig[i] = make_float4(b.x + a.x, b.y + a.y, b.z + a.z, sfun[i]);
}

// P4 over the whole pair set in the pair-once form: the reverse index of the
// tile lists, the pass, and the rows pass that completes every particle's sums.
template <bool COMP>
static int run_forces_po(crk_ctx *ctx, const FRec *fr, const FParams &fp, cudaStream_t s) {
    if (!ctx->lists_valid) return crk_set_error(ctx, CRK_ESTATE, "P4 forces: neighbour lists are not built");
    int rc = crk_ensure_pair_once(ctx);
    if (rc) return rc;
    typename P4PO<COMP>::Params p{fr, ctx->mass, fp, ctx->acc, ctx->vq, ctx->Fst, ctx->po_rowA, ctx->po_rowB};
    prof_begin(ctx, PROF_P4, s);
    k_po_rev<<<grid_for(ctx->ntiles, 8), 256, 0, s>>>(ctx->ntiles, ctx->uofs, ctx->ulist, ctx->po_rev,
                                                       ctx->po_self, ctx->po_tofs, ctx->po_tlist,
                                                       ctx->counters + CNT_PO_MISS);
    k_po<P4PO<COMP>><<<grid_for(ctx->ntiles, PO_WARPS), PO_WARPS * 32, 0, s>>>(po_geom(ctx), p);
    k_p4po_rows<COMP><<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->po_tofs, ctx->po_self, ctx->po_rowA,
                                                            ctx->po_rowB, ctx->mass, fp, ctx->acc, ctx->vq);
    ctx->launches += 3;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, "P4 forces (pair-once)");
    ctx->fst_po = 1;
    return CRK_OK;
}

// P5 over the pair-once stored forces: the pass and its rows pass.
template <bool COMP, bool DUAL>
static int run_compat_po(crk_ctx *ctx, const float4 *sig, float ia4, const unsigned long long *skip, float *du2,
                         cudaStream_t s, const char *what) {
    if (!ctx->lists_valid) return crk_set_error(ctx, CRK_ESTATE, "%s: neighbour lists are not built", what);
    typename P5PO<COMP, DUAL>::Params p{sig, ctx->Fst, ctx->mass, ctx->du, ia4, skip, du2, ctx->po_rowB};
    prof_begin(ctx, PROF_P5, s);
    k_po<P5PO<COMP, DUAL>><<<grid_for(ctx->ntiles, PO_WARPS), PO_WARPS * 32, 0, s>>>(po_geom(ctx), p);
    k_p5po_rows<COMP, DUAL><<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->po_tofs, ctx->po_self, ctx->po_rowB,
                                                                  ctx->mass, ia4, skip, ctx->du, du2);
    ctx->launches += 2;
    prof_end(ctx, s);
    CRK_LAUNCH_CHECK(ctx, what);
    return CRK_OK;
}

// Which form P5 takes: that of the P4 whose forces it reads.
static int p5_form(crk_ctx *ctx, bool *po) {
    *po = ctx->fst_po != 0;
    if (*po && ctx->act)
        return crk_set_error(ctx, CRK_ESTATE, "P5 over a tile subset needs the directed form of the stored forces");
    return CRK_OK;
}

int run_forces(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    FParams fp = fparams(ctx->p);
    if (ctx->p.density) {   // the RK-corrected density of the current corrections
        int rc = run_density(ctx, s);
        if (rc) return rc;
    }
    FSrc src{ctx->q4, ctx->hs, ctx->p.density ? ctx->rho : nullptr, ctx->V, ctx->vel, ctx->mass, ctx->corr,
             ctx->gv};
    k_pack_frec<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, src, fp, reinterpret_cast<FRec *>(ctx->frec),
                                                     ctx->sfun);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "pack pair records");
    const FRec *fr = reinterpret_cast<const FRec *>(ctx->frec);
    if (!ctx->act && ctx->p.pair_form == 1)
        return ctx->p.precision >= 1 ? run_forces_po<true>(ctx, fr, fp, s) : run_forces_po<false>(ctx, fr, fp, s);
    ctx->fst_po = 0;
    if (ctx->p.precision >= 1) {
        typename P4<true>::Params p{fr, ctx->mass, fp, ctx->acc, ctx->vq, ctx->Fst};
        return launch_lpass<P4<true>, 1>(ctx, PROF_P4, p, s, "P4 forces");
    }
    typename P4<false>::Params p{fr, ctx->mass, fp, ctx->acc, ctx->vq, ctx->Fst};
    return launch_lpass<P4<false>, 1>(ctx, PROF_P4, p, s, "P4 forces");
}

// P5 for the kick vb -> va (sorted float4 arrays), with the F_ij of the last P4;
// skip (device flag, may be null) makes the pass read nothing when set.
int run_compatible(crk_ctx *ctx, cudaStream_t s, const unsigned long long *skip) {
    if (ctx->n == 0) return CRK_OK;
    k_sig<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->vb, ctx->va, ctx->sfun, ctx->sig);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "kick sums");
    const float ia4 = (float)(1.0 / (ctx->p.a * ctx->p.a * ctx->p.a * ctx->p.a));
    bool po = false;
    int rc = p5_form(ctx, &po);
    if (rc) return rc;
    if (po)
        return ctx->p.precision >= 1
                   ? run_compat_po<true, false>(ctx, ctx->sig, ia4, skip, nullptr, s, "P5 compatible energy")
                   : run_compat_po<false, false>(ctx, ctx->sig, ia4, skip, nullptr, s, "P5 compatible energy");
    if (ctx->p.precision >= 1) {
        typename P5<true>::Params p{ctx->sig, ctx->Fst, ctx->mass, ctx->du, ia4, skip, nullptr};
        return launch_lpass<P5<true>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy");
    }
    typename P5<false>::Params p{ctx->sig, ctx->Fst, ctx->mass, ctx->du, ia4, skip, nullptr};
    return launch_lpass<P5<false>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy");
}

// kick sums of this closing kick (vb -> va) and of the next step's opening
// kick (vb' = p1 = va, va' = p1 + a dt'/2 with the next step's dt, as k_kick1
// will form them), side by side: sig2[2i] = sig_i, sig2[2i+1] = sig'_i
__global__ void k_sig_dual(int n, const double *dtn, const int32_t *__restrict__ sbox,
                           const float4 *__restrict__ vb, const float4 *__restrict__ va,
                           const float4 *__restrict__ acc, const float *__restrict__ sfun, float4 *__restrict__ sig2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h = (float)(0.5 * dtn[sbox ? sbox[i] : 0]);
    float4 b = vb[i], v = va[i], a = acc[i];
    const float sf = sfun[i];
    sig2[2 * (size_t)i] = make_float4(b.x + v.x, b.y + v.y, b.z + v.z, sf);
    sig2[2 * (size_t)i + 1] = make_float4(v.x + fmaf(h, a.x, v.x), v.y + fmaf(h, a.y, v.y), v.z + fmaf(h, a.z, v.z), sf);
}

// P5 of this closing kick (vb -> va into du) and of the next step's opening
// kick (its dt per box in dtn; into du_next) in one pass over the stored forces.
int run_compatible_dual(crk_ctx *ctx, const double *dtn, const int32_t *sbox, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    k_sig_dual<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, dtn, sbox, ctx->vb, ctx->va, ctx->acc, ctx->sfun,
                                                      ctx->sig2);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "kick sums");
    const float ia4 = (float)(1.0 / (ctx->p.a * ctx->p.a * ctx->p.a * ctx->p.a));
    bool po = false;
    int rc = p5_form(ctx, &po);
    if (rc) return rc;
    if (po)
        return ctx->p.precision >= 1 ? run_compat_po<true, true>(ctx, ctx->sig2, ia4, nullptr, ctx->du_next, s,
                                                                 "P5 compatible energy (two kicks)")
                                     : run_compat_po<false, true>(ctx, ctx->sig2, ia4, nullptr, ctx->du_next, s,
                                                                  "P5 compatible energy (two kicks)");
    if (ctx->p.precision >= 1) {
        typename P5<true, true>::Params p{ctx->sig2, ctx->Fst, ctx->mass, ctx->du, ia4, nullptr, ctx->du_next};
        return launch_lpass<P5<true, true>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy (two kicks)",
                                              TUNE_P5_DUAL);
    }
    typename P5<false, true>::Params p{ctx->sig2, ctx->Fst, ctx->mass, ctx->du, ia4, nullptr, ctx->du_next};
    return launch_lpass<P5<false, true>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy (two kicks)",
                                              TUNE_P5_DUAL);
}

}  // namespace crk
