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
};

// Per-particle record of the pair-set passes (160 bytes).
struct __align__(32) FRec {
    uint4 q;        // qx, qy, qz, H
    float4 k0;      // 1/h, cW = 495/(32 pi h^3), cG = -1155/(4 pi h^5), h_hat = h/n_h
    float4 k1;      // V, P, rho, c_s
    float4 k2;      // vx, vy, vz, A
    float4 k3;      // Bx, By, Bz, gAx
    float4 k4;      // gAy, gAz, gB00, gB01
    float4 k5;      // gB02, gB10, gB11, gB12
    float4 k6;      // gB20, gB21, gB22, gv00
    float4 k7;      // gv01, gv02, gv10, gv11
    float4 k8;      // gv12, gv20, gv21, gv22
};

struct FSrc {
    const uint4 *q4;
    const float *hs;
    const float *V;
    const float4 *vel;
    const float *mass;
    const CorrRec *corr;
    const GvRec *gv;
};

__device__ __forceinline__ FRec load_frec(int j, const FSrc &src, const FParams &fp) {
    FRec r;
    r.q = src.q4[j];
    float h = src.hs[j], ih = 1.f / h, ih2 = ih * ih, ih3 = ih2 * ih;
    r.k0 = make_float4(ih, KW * ih3, -KG * ih3 * ih2, h * fp.inv_nh);
    float V = src.V[j];
    float4 v = src.vel[j];
    float rho = src.mass[j] / V;
    float P = fp.gm1 * rho * v.w;
    r.k1 = make_float4(V, P, rho, sqrtf(fmaxf(fp.gamma * P / rho, 0.f)));
    CorrRec c = src.corr[j];
    GvRec g = src.gv[j];
    r.k2 = make_float4(v.x, v.y, v.z, c.c0.x);
    r.k3 = make_float4(c.c0.y, c.c0.z, c.c0.w, c.c1.x);
    r.k4 = make_float4(c.c1.y, c.c1.z, c.c1.w, c.c2.x);
    r.k5 = make_float4(c.c2.y, c.c2.z, c.c2.w, c.c3.x);
    r.k6 = make_float4(c.c3.y, c.c3.z, c.c3.w, g.g0.x);
    r.k7 = make_float4(g.g0.y, g.g0.z, g.g0.w, g.g1.x);
    r.k8 = make_float4(g.g1.y, g.g1.z, g.g1.w, g.g2.x);
    return r;
}

// eq:gRK for particle a with separation x (= x_a - x_b), kernel value W and
// radial factor G (grad W = G x).
__device__ __forceinline__ void grad_rk(const FRec &a, const float x[3], float W, float G, float out[3]) {
    const float A = a.k2.w;
    const float B[3] = {a.k3.x, a.k3.y, a.k3.z};
    const float gA[3] = {a.k3.w, a.k4.x, a.k4.y};
    const float gB[9] = {a.k4.z, a.k4.w, a.k5.x, a.k5.y, a.k5.z, a.k5.w, a.k6.x, a.k6.y, a.k6.z};
    float sB = fmaf(B[0], x[0], fmaf(B[1], x[1], fmaf(B[2], x[2], 1.f)));
    float sW = sB * W, AW = A * W, AsG = A * sB * G;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        float gBx = fmaf(gB[g], x[0], fmaf(gB[3 + g], x[1], gB[6 + g] * x[2]));
        out[g] = fmaf(gA[g], sW, fmaf(AW, gBx + B[g], AsG * x[g]));
    }
}

// grad v . x for particle a
__device__ __forceinline__ void gv_dot(const FRec &a, const float x[3], float o[3]) {
    o[0] = fmaf(a.k6.w, x[0], fmaf(a.k7.x, x[1], a.k7.y * x[2]));
    o[1] = fmaf(a.k7.z, x[0], fmaf(a.k7.w, x[1], a.k8.x * x[2]));
    o[2] = fmaf(a.k8.y, x[0], fmaf(a.k8.z, x[1], a.k8.w * x[2]));
}

__device__ __forceinline__ void kern(const FRec &a, float r, bool in, float &W, float &G) {
    float eta = r * a.k0.x;
    float t = fmaxf(1.f - eta, 0.f);
    float t2 = t * t, t5 = t2 * t2 * t;
    W = in ? a.k0.y * t5 * t * fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f) : 0.f;
    G = in ? a.k0.z * fmaf(5.f, eta, 1.f) * t5 : 0.f;
}

struct PairOut {
    float F[3];    // force on a from b, 1/2 V_a V_b (P~_a + P~_b)(grad W^R_ba - grad W^R_ab)
    float D[3];    // grad W^R_ba - grad W^R_ab
    float Pt_b;    // P_b + Q_b of this pair
    float Q_a;     // Q_a of this pair
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

    // limiter, eq:phi .. eq:phiad
    float pa[3], pb[3];
    gv_dot(a, x, pa);
    gv_dot(b, x, pb);
    float qa = fmaf(x[0], pa[0], fmaf(x[1], pa[1], x[2] * pa[2]));
    float qb = fmaf(x[0], pb[0], fmaf(x[1], pb[1], x[2] * pb[2]));
    float qs = qa + qb;
    float phi = 0.f;
    if (qs != 0.f) {
        float is = FDIV(1.f, qs);
        phi = fminf(fmaxf(4.f * (qa * is) * (qb * is), 0.f), 1.f);
    }
    float eta = fminf(r * a.k0.x, r * b.k0.x);
    if (eta < fp.eta_crit) {
        float e = (eta - fp.eta_crit) * fp.inv_eta_fold;
        phi *= __expf(-e * e);
    }
    // projected velocity difference, eq:hatvi (adot = 0)
    float hp = -0.5f * phi;
    float uh[3];
    uh[0] = fmaf(hp, pa[0] + pb[0], a.k2.x - b.k2.x);
    uh[1] = fmaf(hp, pa[1] + pb[1], a.k2.y - b.k2.y);
    uh[2] = fmaf(hp, pa[2] + pb[2], a.k2.z - b.k2.z);
    float ux = fmaf(uh[0], x[0], fmaf(uh[1], x[1], uh[2] * x[2]));
    // eq:mu, eq:visc
    float hha = a.k0.w, hhb = b.k0.w;
    float mua = fminf(FDIV(hha * ux, fmaf(hha * hha, fp.eps2, r2)), 0.f);
    float mub = fminf(FDIV(hhb * ux, fmaf(hhb * hhb, fp.eps2, r2)), 0.f);
    float Qa = a.k1.z * mua * fmaf(fp.Cq, mua, -fp.Cl * a.k1.w);
    float Qb = b.k1.z * mub * fmaf(fp.Cq, mub, -fp.Cl * b.k1.w);
    float Pta = a.k1.y + Qa, Ptb = b.k1.y + Qb;
    float cF = 0.5f * (a.k1.x * b.k1.x) * (Pta + Ptb);
#pragma unroll
    for (int g = 0; g < 3; g++) o.F[g] = cF * o.D[g];
    o.Pt_b = Ptb;
    o.Q_a = Qa;
}

// Per-particle records of the pair-set passes, packed once per evaluation.
__global__ void k_pack_frec(int n, FSrc src, FParams fp, FRec *__restrict__ out, float *__restrict__ sfun) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    FRec r = load_frec(i, src, fp);
    out[i] = r;
    sfun[i] = r.k1.y / powf(r.k1.z, fp.gamma);       // s = P / rho^gamma (eq:fij)
}

// Two float4 of a record in one 256-bit read-only load (the record is 160 B,
// so every pair of its float4 starts on a 32-byte boundary): one L1 sector
// per lane per instruction instead of half a sector.
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

__device__ __forceinline__ FRec ldg_frec(const FRec *p) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    FRec r;
    float4 a;
    ldg_v8(q, a, r.k0);
    r.q = make_uint4(__float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(a.z), __float_as_uint(a.w));
    ldg_v8(q + 2, r.k1, r.k2);
    ldg_v8(q + 4, r.k3, r.k4);
    ldg_v8(q + 6, r.k5, r.k6);
    ldg_v8(q + 8, r.k7, r.k8);
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
    using Rec = FRec;
    struct Params {
        const FRec *frec;
        const float *mass;
        FParams fp;
        float4 *acc;   // (ax, ay, az, dudt)
        float2 *vq;    // (vsig, qmax)
        float4 *Fst;   // (F_ij, j bits) per list entry
    };
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
            s.me.k0.x = 1.f;
            s.m = 1.f;
        }
        s.vsig = 0.f;
        s.qmax = 0.f;
    }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) { return ldg_frec(p.frec + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &r, uint32_t e, size_t pos, bool in_i, const Params &p) {
        const bool in_j = in_i ? (e >> 31) != 0u : true;
        int dx = (int)(s.me.q.x - r.q.x), dy = (int)(s.me.q.y - r.q.y), dz = (int)(s.me.q.z - r.q.z);
        Sep d = separation(dx, dy, dz);
        float x[3] = {d.x, d.y, d.z};
        PairOut o;
        pair_force(s.me, r, x, d.r2, d.r, in_i, in_j, p.fp, o);
        p.Fst[pos] = make_float4(o.F[0], o.F[1], o.F[2], __uint_as_float(e & 0x3fffffffu));   // F_ij, j
        float dv[3] = {r.k2.x - s.me.k2.x, r.k2.y - s.me.k2.y, r.k2.z - s.me.k2.z};
#pragma unroll
        for (int g = 0; g < 3; g++) s.F[g].add(o.F[g]);
        float wd = fmaf(dv[0], o.D[0], fmaf(dv[1], o.D[1], dv[2] * o.D[2]));
        s.du.add(0.5f * (s.me.k1.x * r.k1.x) * o.Pt_b * wd);
        float vx = -fmaf(dv[0], x[0], fmaf(dv[1], x[1], dv[2] * x[2]));   // (v_i - v_j).x_ij
        if (vx < 0.f && d.r > 0.f) s.vsig = fmaxf(s.vsig, FDIV(-vx, d.r));
        s.qmax = fmaxf(s.qmax, o.Q_a);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        float im = 1.f / s.m;
        p.acc[i] = make_float4(s.F[0].value() * im, s.F[1].value() * im, s.F[2].value() * im, s.du.value() * im);
        p.vq[i] = make_float2(s.vsig, s.qmax);
    }
};

// ================================================================= P5 compatible energy

// sig = (v + v') of the kick and the entropy s of the evaluation state
template <bool COMP>
struct P5 {
    static constexpr bool GATHER = false;
    static constexpr int UNROLL = 3;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    struct Rec {
        float4 sig, F;
    };
    struct Params {
        const float4 *sig;
        const float4 *Fst;
        const float *mass;
        float *du;
    };
    struct IState {
        float4 me;
        float m;
        Acc<COMP> du;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.me = valid ? p.sig[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        s.m = valid ? p.mass[i] : 1.f;
    }
    // the stored entry carries j (written by P4): the list itself is not read
    static constexpr bool ENTRIES = false;
    __device__ static Rec load(uint32_t, size_t pos, const Params &p) {
        const float4 F = __ldg(p.Fst + pos);
        return Rec{__ldg(p.sig + __float_as_uint(F.w)), F};
    }
    __device__ static void pair(IState &s, const Rec &rec, uint32_t, size_t, bool, const Params &) {
        const float4 r = rec.sig;
        const float4 F = rec.F;
        // 2 Delta E_ij = (v_j + v'_j - v_i - v'_i) . F_ij  (reading of eq:Eij)
        float w = fmaf(r.x - s.me.x, F.x, fmaf(r.y - s.me.y, F.y, (r.z - s.me.z) * F.z));
        // eq:fij
        float si = s.me.w, sj = r.w, ss = si + sj;
        float f = 0.5f;
        if (ss != 0.f) {
            bool take_min = (w >= 0.f) == (si >= sj);
            f = (take_min ? fminf(si, sj) : fmaxf(si, sj)) / ss;
        }
        s.du.add(0.5f * f * w);
    }
    __device__ static void finish(IState &s, int i, const Params &p) { p.du[i] = s.du.value() / s.m; }
};

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

int run_forces(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    FParams fp = fparams(ctx->p);
    FSrc src{ctx->q4, ctx->hs, ctx->V, ctx->vel, ctx->mass, ctx->corr, ctx->gv};
    k_pack_frec<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, src, fp, reinterpret_cast<FRec *>(ctx->frec),
                                                     ctx->sfun);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "pack pair records");
    const FRec *fr = reinterpret_cast<const FRec *>(ctx->frec);
    if (ctx->p.precision >= 1) {
        typename P4<true>::Params p{fr, ctx->mass, fp, ctx->acc, ctx->vq, ctx->Fst};
        return launch_lpass<P4<true>, 1>(ctx, PROF_P4, p, s, "P4 forces");
    }
    typename P4<false>::Params p{fr, ctx->mass, fp, ctx->acc, ctx->vq, ctx->Fst};
    return launch_lpass<P4<false>, 1>(ctx, PROF_P4, p, s, "P4 forces");
}

// P5 for the kick vb -> va (sorted float4 arrays), with the F_ij of the last P4.
int run_compatible(crk_ctx *ctx, cudaStream_t s) {
    if (ctx->n == 0) return CRK_OK;
    k_sig<<<grid_for(ctx->n, 256), 256, 0, s>>>(ctx->n, ctx->vb, ctx->va, ctx->sfun, ctx->sig);
    ++ctx->launches;
    CRK_LAUNCH_CHECK(ctx, "kick sums");
    if (ctx->p.precision >= 1) {
        typename P5<true>::Params p{ctx->sig, ctx->Fst, ctx->mass, ctx->du};
        return launch_lpass<P5<true>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy");
    }
    typename P5<false>::Params p{ctx->sig, ctx->Fst, ctx->mass, ctx->du};
    return launch_lpass<P5<false>, 8>(ctx, PROF_P5, p, s, "P5 compatible energy");
}

}  // namespace crk
