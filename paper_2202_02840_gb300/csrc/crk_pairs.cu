// crk_pairs.cu -- gather pair passes over gather(i) = {j : |dq|^2 < H_i^2},
// walking each particle's neighbour list (P1 volumes are fused into the
// list-counting walk, crk_walk.cu):
//   P2 RK corrections    (Sec. 1.2 eq:RK, eq:gRK, moment conditions)
//   P3 velocity gradient (Sec. 1.2 eq:gradv)
// plus the tile-walk neighbour-set inspection pass.
#include "crk_pass.cuh"

namespace crk {

// ================================================================= neighbour sets

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

template <bool UNION>
struct PN {
    struct Params {
        const uint4 *q4;
        const int32_t *perm;
        const int32_t *sbox;   // batched boxes (null: one box)
        int32_t *cnt;
        uint32_t *hash;
    };
    struct __align__(16) JRec {
        uint4 q;
        int4 id;   // caller index, box, -, -
    };
    struct IState {
        uint4 q;
        unsigned long long H2;
        int c, box;
        uint32_t h;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        s.H2 = (unsigned long long)s.q.w * s.q.w;
        s.c = 0;
        s.box = (valid && p.sbox) ? p.sbox[i] : 0;
        s.h = 0u;
    }
    __device__ static void stage(JRec &r, int j, const Params &p) {
        r.q = p.q4[j];
        r.id = make_int4(p.perm[j], p.sbox ? p.sbox[j] : 0, 0, 0);
    }
    __device__ static void pair(IState &s, const JRec &r, int j, int i, bool valid, const Params &) {
        int dx = (int)(s.q.x - r.q.x), dy = (int)(s.q.y - r.q.y), dz = (int)(s.q.z - r.q.z);
        unsigned long long R2 = r.id.y == s.box ? r2_fixed(dx, dy, dz) : ~0ull;
        bool in;
        if (UNION) {
            unsigned long long Hj2 = (unsigned long long)r.q.w * r.q.w;
            in = valid && i != j && (R2 < s.H2 || R2 < Hj2);
        } else {
            in = R2 < s.H2;
        }
        if (in) {
            s.c++;
            s.h += fmix32((uint32_t)r.id.x + 1u);
        }
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        p.cnt[i] = s.c;
        p.hash[i] = s.h;
    }
    __device__ static int count(const IState &) { return 0; }
};

int run_neighbours(crk_ctx *ctx, int mode, int32_t *cnt, uint32_t *hash, cudaStream_t s) {
    if (mode == 0) {
        PN<false>::Params p{ctx->q4, ctx->perm, ctx->nbox > 1 ? ctx->sbox : nullptr, cnt, hash};
        return launch_pass<PN<false>, 8>(ctx, PROF_PN, true, p, nullptr, s, "neighbour sets");
    }
    PN<true>::Params p{ctx->q4, ctx->perm, ctx->nbox > 1 ? ctx->sbox : nullptr, cnt, hash};
    return launch_pass<PN<true>, 8>(ctx, PROF_PN, true, p, nullptr, s, "neighbour sets");
}

// ================================================================= P2 corrections

// symmetric index of (a,b): xx, xy, xz, yy, yz, zz
__host__ __device__ constexpr int sym(int a, int b) {
    return a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5));
}

// symmetric index of (a,b,c): xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz
__host__ __device__ constexpr int sym3(int a, int b, int c) {
    const int lo = a < b ? (a < c ? a : c) : (b < c ? b : c);
    const int hi = a > b ? (a > c ? a : c) : (b > c ? b : c);
    const int mid = a + b + c - lo - hi;
    return lo == 0 ? (mid == 0 ? hi : (mid == 1 ? 2 + hi : 5)) : (lo == 1 ? (mid == 1 ? 5 + hi : 8) : 9);
}

// Solve the RK coefficients from the moments (derived from the two moment
// conditions of Sec. 1.2):  B = -m2^-1 m1, A = 1/(m0 + m1.B),
// d_g B = -m2^-1 (d_g m1 + (d_g m2) B), d_g A = -A^2 (d_g m0 + B.d_g m1 + m1.d_g B).
// dm1[a*3+g] = d_g m1^a, dm2[sym(a,b)*3+g] = d_g m2^ab.
template <typename T, typename I>
__device__ __forceinline__ void rk_solve(I m0f, const I *m1f, const I *m2f, const I *dm0f,
                                         const I *dm1f, const I *dm2f, CorrRec &out) {
    T m[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) m[3 * a + b] = (T)m2f[sym(a, b)];
    T c00 = m[4] * m[8] - m[5] * m[7];
    T c01 = m[5] * m[6] - m[3] * m[8];
    T c02 = m[3] * m[7] - m[4] * m[6];
    T det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    T id = (T)1 / det;
    T mi[9];
    mi[0] = c00 * id;
    mi[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    mi[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    mi[3] = c01 * id;
    mi[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    mi[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    mi[6] = c02 * id;
    mi[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    mi[8] = (m[0] * m[4] - m[1] * m[3]) * id;
    T m1[3] = {(T)m1f[0], (T)m1f[1], (T)m1f[2]};
    T B[3];
#pragma unroll
    for (int a = 0; a < 3; a++) B[a] = -(mi[3 * a] * m1[0] + mi[3 * a + 1] * m1[1] + mi[3 * a + 2] * m1[2]);
    T A = (T)1 / ((T)m0f + m1[0] * B[0] + m1[1] * B[1] + m1[2] * B[2]);
    T dB[9];
#pragma unroll
    for (int g = 0; g < 3; g++) {
        T rhs[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            T r = (T)dm1f[3 * a + g];
#pragma unroll
            for (int b = 0; b < 3; b++) r += (T)dm2f[3 * sym(a, b) + g] * B[b];
            rhs[a] = r;
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
            dB[3 * a + g] = -(mi[3 * a] * rhs[0] + mi[3 * a + 1] * rhs[1] + mi[3 * a + 2] * rhs[2]);
    }
    T dA[3];
#pragma unroll
    for (int g = 0; g < 3; g++) {
        T acc = (T)dm0f[g];
#pragma unroll
        for (int a = 0; a < 3; a++) acc += B[a] * (T)dm1f[3 * a + g] + m1[a] * dB[3 * a + g];
        dA[g] = -A * A * acc;
    }
    out.c0 = make_float4((float)A, (float)B[0], (float)B[1], (float)B[2]);
    out.c1 = make_float4((float)dA[0], (float)dA[1], (float)dA[2], (float)dB[0]);
    out.c2 = make_float4((float)dB[1], (float)dB[2], (float)dB[3], (float)dB[4]);
    out.c3 = make_float4((float)dB[5], (float)dB[6], (float)dB[7], (float)dB[8]);
}

// The pair sums of P2 (unnormalised: W-type sums without 495/(32 pi h^3),
// gradient sums without 1155/(4 pi h^5)): m0 = sum V Wu, m1 = sum V x Wu,
// m2 = sum V x x Wu (6 distinct), dm0 = sum V x Gu, s1 = sum V x^a x^g Gu (6),
// s2 = sum V x^a x^b x^g Gu (10), with grad W = 1155/(4 pi h^5) Gu x.
template <typename T>
struct PairSums {
    T m0, m1[3], m2[6], dm0[3], s1[6], s2[10];
};

// Moments from the pair sums: W-type sums scale by cW = 495/(32 pi h^3),
// gradient sums by cG = 1155/(4 pi h^5); then
//   d_g m1^a = delta_ag m0 + cG sum V x^a x^g Gu,
//   d_g m2^ab = delta_ag m1^b + delta_bg m1^a + cG sum V x^a x^b x^g Gu.
// The diagonal of d m1 nearly cancels (sum V x^a d_a W ~ -m0), so the mixed
// paths form every moment in FP64 from the (compensated) sums and FP64
// constants before that cancellation.
template <typename T>
__device__ __forceinline__ void moments(float h, const PairSums<T> &s, T &m0, T *m1, T *m2, T *dm0, T *dm1,
                                        T *dm2) {
    T ih = (T)1 / (T)h, ih2 = ih * ih, ih3 = ih2 * ih;
    T cW = (T)KW_D * ih3;         // 495 / (32 pi)
    T cG = (T)KG_D * ih3 * ih2;   // 1155 / (4 pi)
    m0 = cW * s.m0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        m1[a] = cW * s.m1[a];
        dm0[a] = cG * s.dm0[a];
    }
#pragma unroll
    for (int q = 0; q < 6; q++) m2[q] = cW * s.m2[q];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int g = 0; g < 3; g++) dm1[3 * a + g] = cG * s.s1[sym(a, g)] + (a == g ? m0 : (T)0);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = a; b < 3; b++)
#pragma unroll
            for (int g = 0; g < 3; g++) {
                int q = sym(a, b);
                T v = cG * s.s2[sym3(a, b, g)];
                if (a == g) v += m1[b];
                if (b == g) v += m1[a];
                dm2[3 * q + g] = v;
            }
}

template <bool FP64_SOLVE, bool COMP>
struct P2 {
    static constexpr bool GATHER = true;
    static constexpr int UNROLL = 4;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    using Rec = uint4;
    struct Params {
        const uint4 *q4;
        const uint4 *qV;   // (qx, qy, qz, V bits)
        const float *hs;
        CorrRec *corr;
    };
    struct IState {
        uint4 q;
        float h, inv_h;
        // s1 = sum V x^a x^g Gu and s2 = sum V x^a x^b x^g Gu are symmetric
        // tensors: only their distinct components are summed
        Acc<COMP> m0, m1[3], m2[6], dm0[3], s1[6], s2[10];
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        s.h = valid ? p.hs[i] : 1.f;
        s.inv_h = 1.f / s.h;
        s.m0 = Acc<COMP>();
#pragma unroll
        for (int a = 0; a < 3; a++) s.m1[a] = s.dm0[a] = Acc<COMP>();
#pragma unroll
        for (int a = 0; a < 6; a++) s.m2[a] = Acc<COMP>();
#pragma unroll
        for (int a = 0; a < 6; a++) s.s1[a] = Acc<COMP>();
#pragma unroll
        for (int a = 0; a < 10; a++) s.s2[a] = Acc<COMP>();
        // self term of gather(i): x = 0, W(0) (unnormalised 1), grad W(0) = 0
        if (valid) s.m0.add(__uint_as_float(__ldg(&p.qV[i].w)));
    }
    __device__ static void zero(IState &s) {
        s.m0 = Acc<COMP>();
        for (int a = 0; a < 3; a++) s.m1[a] = s.dm0[a] = Acc<COMP>();
        for (int a = 0; a < 6; a++) s.m2[a] = Acc<COMP>();
        for (int a = 0; a < 6; a++) s.s1[a] = Acc<COMP>();
        for (int a = 0; a < 10; a++) s.s2[a] = Acc<COMP>();
    }
    __device__ static void merge(IState &s, const IState &o) {
        merge_acc(s.m0, o.m0);
        for (int a = 0; a < 3; a++) {
            merge_acc(s.m1[a], o.m1[a]);
            merge_acc(s.dm0[a], o.dm0[a]);
        }
        for (int a = 0; a < 6; a++) merge_acc(s.m2[a], o.m2[a]);
        for (int a = 0; a < 6; a++) merge_acc(s.s1[a], o.s1[a]);
        for (int a = 0; a < 10; a++) merge_acc(s.s2[a], o.s2[a]);
    }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) { return __ldg(p.qV + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &r, uint32_t, size_t, bool, const Params &) {
        int dx = (int)(s.q.x - r.x), dy = (int)(s.q.y - r.y), dz = (int)(s.q.z - r.z);
        const float Vj = __uint_as_float(r.w);
        Sep d = separation(dx, dy, dz);
        float x[3] = {d.x, d.y, d.z};
        float eta = d.r * s.inv_h;
        float t = fmaxf(1.f - eta, 0.f);
        float t2 = t * t, t4 = t2 * t2, t5 = t4 * t;
        float Wu = t5 * t * fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f);   // W / (495/(32 pi h^3))
        float Gu = -fmaf(5.f, eta, 1.f) * t5;                        // grad W / (1155/(4 pi h^5) x)
        float w = Vj * Wu, g = Vj * Gu;
        float gx[3] = {g * x[0], g * x[1], g * x[2]};
        float xx[6] = {x[0] * x[0], x[0] * x[1], x[0] * x[2], x[1] * x[1], x[1] * x[2], x[2] * x[2]};
        s.m0.add(w);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            s.m1[a].add(w * x[a]);
            s.dm0[a].add(gx[a]);
        }
#pragma unroll
        for (int q = 0; q < 6; q++) s.m2[q].add(w * xx[q]);
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = a; b < 3; b++) {
                s.s1[sym(a, b)].add(x[a] * gx[b]);
#pragma unroll
                for (int gg = b; gg < 3; gg++) s.s2[sym3(a, b, gg)].add(xx[sym(a, b)] * gx[gg]);
            }
    }
    // Moments from the pair sums: W-type sums scale by cW = 495/(32 pi h^3),
    // gradient sums by cG = 1155/(4 pi h^5); then
    //   d_g m1^a = delta_ag m0 + cG sum V x^a x^g Gu,
    //   d_g m2^ab = delta_ag m1^b + delta_bg m1^a + cG sum V x^a x^b x^g Gu.
    // The diagonal of d m1 nearly cancels (sum V x^a d_a W ~ -m0), so the mixed
    // path forms every moment in FP64 from the compensated (hi, lo) sums and
    // FP64 constants before that cancellation.
    __device__ static void finish(IState &s, int i, const Params &p) {
        CorrRec out;
        auto val = [](const Acc<COMP> &a) -> double { return COMP ? (double)a.s - (double)a.c : (double)a.s; };
        if (FP64_SOLVE) {
            PairSums<double> ps;
            ps.m0 = val(s.m0);
            for (int a = 0; a < 3; a++) ps.m1[a] = val(s.m1[a]), ps.dm0[a] = val(s.dm0[a]);
            for (int q = 0; q < 6; q++) ps.m2[q] = val(s.m2[q]), ps.s1[q] = val(s.s1[q]);
            for (int q = 0; q < 10; q++) ps.s2[q] = val(s.s2[q]);
            double m0, m1[3], m2[6], dm0[3], dm1[9], dm2[18];
            moments<double>(s.h, ps, m0, m1, m2, dm0, dm1, dm2);
            rk_solve<double, double>(m0, m1, m2, dm0, dm1, dm2, out);
        } else {
            PairSums<float> ps;
            ps.m0 = s.m0.value();
            for (int a = 0; a < 3; a++) ps.m1[a] = s.m1[a].value(), ps.dm0[a] = s.dm0[a].value();
            for (int q = 0; q < 6; q++) ps.m2[q] = s.m2[q].value(), ps.s1[q] = s.s1[q].value();
            for (int q = 0; q < 10; q++) ps.s2[q] = s.s2[q].value();
            float m0, m1[3], m2[6], dm0[3], dm1[9], dm2[18];
            moments<float>(s.h, ps, m0, m1, m2, dm0, dm1, dm2);
            rk_solve<float, float>(m0, m1, m2, dm0, dm1, dm2, out);
        }
        p.corr[i] = out;
    }
};

// ---------------------------------------------------------------- P2 in float-float (precision 3)
//
// On lattice-like neighbourhoods the odd moments, grad m0, and the diagonal of
// grad m1 = delta m0 + sum V x grad W cancel to ~1e-4 of their terms, so the
// result keeps only ~1e-4 of the terms' relative accuracy: FP32 pair terms
// (x rounded to FP32, t = 1 - eta rounded and raised to the sixth power, each
// product rounded) leave 1e-5 .. 3e-5 of the field RMS in B, grad A, grad B.
// This form carries every pair term as an unevaluated sum hi + lo of two
// floats (an error-free product hi = a b, lo = fma(a, b, -hi), plus the
// operands' own lo parts to first order), starting from exact inputs: the
// separation x = dq 2^-32 split exactly into a float and its integer residual,
// r = sqrt(R^2) from the exact integer R^2 with one Newton correction, eta
// = r / h with its division residual, and t = 1 - eta by an exact
// Fast2Sum.  The hi parts are summed by TwoSum, their rounding errors and the
// lo parts in plain FP32 (they are ~1e-7 of the terms, so their own rounding
// is negligible); each moment is then hi + lo in FP64.  Only FP32
// arithmetic runs per pair; the __f*_rn intrinsics keep the compiler from
// fusing the products whose rounding errors are being captured.
struct FF {
    float hi, lo;
};
constexpr float K35_3_LO = (float)(35.0 / 3.0 - (double)K35_3);   // 35/3 - K35_3

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);                     // exact: a.hi b.hi - p
    return FF{p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e))};
}

__device__ __forceinline__ FF ff_add(FF a, float b) {      // TwoSum of a.hi + b, lo carried
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return FF{s, e + a.lo};
}

// x = d 2^-32 exactly: hi = the float nearest d (times 2^-32), lo = the integer
// residual (|residual| <= 2^6 for |d| < 2^31) times 2^-32
__device__ __forceinline__ FF ff_coord(int d) {
    const float f = __int2float_rn(d);
    const int back = __float2int_rz(f);
    return FF{f * TWO_M32, __int2float_rn(d - back) * TWO_M32};
}

// accumulator of FF terms: each hi part is added by TwoSum, whose exact
// rounding error joins the lo parts in a plain FP32 sum.  (Kahan's
// compensation is exact only while the running sum outweighs the term, which
// the cancelling moment sums violate: it left ~2e-6 of the RMS in B.)
struct AccFF {
    float s = 0.f, l = 0.f;
    __device__ __forceinline__ void add(FF v) {
        const float t = __fadd_rn(s, v.hi);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v.hi, bp));
        s = t;
        l += e + v.lo;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)l; }
};

__device__ __forceinline__ void merge_acc(AccFF &d, const AccFF &o) { d.add(FF{o.s, o.l}); }

struct P2X {
    static constexpr bool GATHER = true;
    static constexpr int UNROLL = 2;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    static constexpr bool NOTUNE = true;   // one accuracy mode, one loop form
    using Rec = uint4;
    using Params = P2<true, true>::Params;
    struct IState {
        uint4 q;
        float h;
        FF ih;                                  // 1/h as hi + lo
        AccFF m0, m1[3], m2[6], dm0[3], s1[6], s2[10];
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        s.h = valid ? p.hs[i] : 1.f;
        const float ih = __frcp_rn(s.h);
        s.ih = FF{ih, __fmul_rn(fmaf(-ih, s.h, 1.f), ih)};   // 1/h - ih to first order
        s.m0 = AccFF();
        for (int a = 0; a < 3; a++) s.m1[a] = s.dm0[a] = AccFF();
        for (int a = 0; a < 6; a++) s.m2[a] = s.s1[a] = AccFF();
        for (int a = 0; a < 10; a++) s.s2[a] = AccFF();
        if (valid) s.m0.add(FF{__uint_as_float(__ldg(&p.qV[i].w)), 0.f});   // self: W(0) unnormalised 1
    }
    __device__ static void zero(IState &s) {
        s.m0 = AccFF();
        for (int a = 0; a < 3; a++) s.m1[a] = s.dm0[a] = AccFF();
        for (int a = 0; a < 6; a++) s.m2[a] = s.s1[a] = AccFF();
        for (int a = 0; a < 10; a++) s.s2[a] = AccFF();
    }
    __device__ static void merge(IState &s, const IState &o) {
        merge_acc(s.m0, o.m0);
        for (int a = 0; a < 3; a++) merge_acc(s.m1[a], o.m1[a]), merge_acc(s.dm0[a], o.dm0[a]);
        for (int a = 0; a < 6; a++) merge_acc(s.m2[a], o.m2[a]), merge_acc(s.s1[a], o.s1[a]);
        for (int a = 0; a < 10; a++) merge_acc(s.s2[a], o.s2[a]);
    }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) { return __ldg(p.qV + (e & 0x3fffffffu)); }
    __device__ static void pair(IState &s, const Rec &rc, uint32_t, size_t, bool, const Params &) {
        const int dx = (int)(s.q.x - rc.x), dy = (int)(s.q.y - rc.y), dz = (int)(s.q.z - rc.z);
        const float Vj = __uint_as_float(rc.w);
        const FF x[3] = {ff_coord(dx), ff_coord(dy), ff_coord(dz)};
        // r 2^32 = sqrt(R^2), R^2 exact; hi correctly rounded, lo from one Newton step
        const unsigned long long R2 = r2_fixed(dx, dy, dz);
        const float R2h = __ull2float_rn(R2);
        const float R2l = __ll2float_rn((long long)(R2 - __float2ull_rz(R2h)));
        const float rh = __fsqrt_rn(R2h);
        const float rl = rh > 0.f ? __fdividef(fmaf(-rh, rh, R2h) + R2l, 2.f * rh) : 0.f;
        // eta = r / h: hi = rounded product, lo = its residual plus the lo parts
        const FF r = FF{rh * TWO_M32, rl * TWO_M32};
        const FF eta = ff_mul(r, s.ih);
        // t = 1 - eta: Fast2Sum (|1| >= eta) gives the exact residual of 1 - eta.hi
        const float th = __fsub_rn(1.f, eta.hi);
        const float tr = __fsub_rn(__fsub_rn(th, 1.f), -eta.hi);   // (1 - eta.hi) - th, negated
        const FF t = FF{th, -tr - eta.lo};
        const FF t2 = ff_mul(t, t), t4 = ff_mul(t2, t2), t5 = ff_mul(t4, t), t6 = ff_mul(t5, t);
        // poly = 1 + eta (6 + eta 35/3), with 35/3 as the float K35_3 plus its residual
        const FF poly = ff_add(ff_mul(ff_add(ff_mul(eta, FF{K35_3, K35_3_LO}), 6.f), eta), 1.f);
        const FF Wu = ff_mul(t6, poly);                              // W / (495/(32 pi h^3))
        const FF g5 = ff_add(ff_mul(eta, FF{5.f, 0.f}), 1.f);
        const FF Gn = ff_mul(t5, g5);                                // -grad W / (1155/(4 pi h^5) x)
        const FF w = ff_mul(FF{Vj, 0.f}, Wu);
        const FF gn = ff_mul(FF{Vj, 0.f}, Gn);
        const FF gx[3] = {ff_mul(gn, x[0]), ff_mul(gn, x[1]), ff_mul(gn, x[2])};
        s.m0.add(w);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            s.m1[a].add(ff_mul(w, x[a]));
            s.dm0[a].add(FF{-gx[a].hi, -gx[a].lo});
        }
        // m2 and s2 in float-float too: where m2 is nearly singular along a
        // direction no axis shares (a tilted sheet or filament, cond ~1e6) its
        // FP32 rounding is amplified cond-fold in B and grad B
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = a; b < 3; b++) {
                const FF xab = ff_mul(x[a], x[b]);
                s.m2[sym(a, b)].add(ff_mul(w, xab));
                const FF sx = ff_mul(x[a], gx[b]);
                s.s1[sym(a, b)].add(FF{-sx.hi, -sx.lo});
#pragma unroll
                for (int gg = b; gg < 3; gg++) {
                    const FF v = ff_mul(xab, gx[gg]);
                    s.s2[sym3(a, b, gg)].add(FF{-v.hi, -v.lo});
                }
            }
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        PairSums<double> ps;
        ps.m0 = s.m0.value();
        for (int a = 0; a < 3; a++) ps.m1[a] = s.m1[a].value(), ps.dm0[a] = s.dm0[a].value();
        for (int q = 0; q < 6; q++) ps.m2[q] = s.m2[q].value(), ps.s1[q] = s.s1[q].value();
        for (int q = 0; q < 10; q++) ps.s2[q] = s.s2[q].value();
        double m0, m1[3], m2[6], dm0[3], dm1[9], dm2[18];
        moments<double>(s.h, ps, m0, m1, m2, dm0, dm1, dm2);
        CorrRec out;
        rk_solve<double, double>(m0, m1, m2, dm0, dm1, dm2, out);
        p.corr[i] = out;
    }
};

// ================================================================= P3 grad v

template <bool COMP>
struct P3 {
    static constexpr bool GATHER = true;
    static constexpr int UNROLL = 3;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    struct Params {
        const uint4 *q4;
        const uint4 *qV;
        const float *hs;
        const float4 *vel;
        const CorrRec *corr;
        GvRec *gv;
        float inv_a;        // the state holds p = a v: grad v = (1/a) grad p
    };
    struct IState {
        uint4 q;
        float inv_h, cW, cG;
        float A, B[3], gA[3], gB[9], v[3];
        Acc<COMP> acc[9];
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        float h = valid ? p.hs[i] : 1.f;
        s.inv_h = 1.f / h;
        float ih2 = s.inv_h * s.inv_h, ih3 = ih2 * s.inv_h;
        s.cW = KW * ih3;
        s.cG = -KG * ih3 * ih2;
        CorrRec c = valid ? p.corr[i] : CorrRec{};
        float4 v = valid ? p.vel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        s.A = c.c0.x;
        s.B[0] = c.c0.y; s.B[1] = c.c0.z; s.B[2] = c.c0.w;
        s.gA[0] = c.c1.x; s.gA[1] = c.c1.y; s.gA[2] = c.c1.z;
        s.gB[0] = c.c1.w; s.gB[1] = c.c2.x; s.gB[2] = c.c2.y; s.gB[3] = c.c2.z; s.gB[4] = c.c2.w;
        s.gB[5] = c.c3.x; s.gB[6] = c.c3.y; s.gB[7] = c.c3.z; s.gB[8] = c.c3.w;
        s.v[0] = v.x; s.v[1] = v.y; s.v[2] = v.z;
#pragma unroll
        for (int k = 0; k < 9; k++) s.acc[k] = Acc<COMP>();
    }
    __device__ static void zero(IState &s) {
        for (int k = 0; k < 9; k++) s.acc[k] = Acc<COMP>();
    }
    __device__ static void merge(IState &s, const IState &o) {
        for (int k = 0; k < 9; k++) merge_acc(s.acc[k], o.acc[k]);
    }
    struct Rec {
        uint4 qV;
        float4 v;
    };
    __device__ static Rec load(uint32_t e, size_t, const Params &p) {
        const uint32_t j = e & 0x3fffffffu;
        return Rec{__ldg(p.qV + j), __ldg(p.vel + j)};
    }
    __device__ static void pair(IState &s, const Rec &rec, uint32_t, size_t, bool, const Params &) {
        const uint4 r = rec.qV;
        const float4 vj = rec.v;
        const float Vj = __uint_as_float(r.w);
        int dx = (int)(s.q.x - r.x), dy = (int)(s.q.y - r.y), dz = (int)(s.q.z - r.z);
        Sep d = separation(dx, dy, dz);
        float x[3] = {d.x, d.y, d.z};
        float eta = d.r * s.inv_h;
        float t = fmaxf(1.f - eta, 0.f);
        float t2 = t * t, t4 = t2 * t2, t5 = t4 * t;
        float W = s.cW * t5 * t * fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f);
        float G = s.cG * fmaf(5.f, eta, 1.f) * t5;       // grad W = G x
        // eq:gRK with the i-side coefficients
        float sB = fmaf(s.B[0], x[0], fmaf(s.B[1], x[1], fmaf(s.B[2], x[2], 1.f)));
        float sW = sB * W, AW = s.A * W, AsG = s.A * sB * G;
        float gR[3];
#pragma unroll
        for (int g = 0; g < 3; g++) {
            float gBx = fmaf(s.gB[g], x[0], fmaf(s.gB[3 + g], x[1], s.gB[6 + g] * x[2]));
            gR[g] = fmaf(s.gA[g], sW, fmaf(AW, gBx + s.B[g], AsG * x[g]));
        }
        float Vd[3] = {Vj * (s.v[0] - vj.x), Vj * (s.v[1] - vj.y), Vj * (s.v[2] - vj.z)};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) s.acc[3 * a + b].add(-Vd[a] * gR[b]);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        GvRec g;
        const float k = p.inv_a;
        g.g0 = make_float4(s.acc[0].value() * k, s.acc[1].value() * k, s.acc[2].value() * k, s.acc[3].value() * k);
        g.g1 = make_float4(s.acc[4].value() * k, s.acc[5].value() * k, s.acc[6].value() * k, s.acc[7].value() * k);
        g.g2 = make_float4(s.acc[8].value() * k, 0.f, 0.f, 0.f);
        p.gv[i] = g;
    }
};

// ================================================================= RK-corrected density

// crk_params.density = 1: rho_i = sum over gather(i), self included, of
// m_j W^R_ij = A_i (1 + B_i . x_ij) W(r_ij, h_i) (eq:RK): the RK interpolant of
// m_j / V_j, exact for constant and linear fields.
struct PD {
    static constexpr bool GATHER = true;
    static constexpr int UNROLL = 4;
    static constexpr bool ENTRIES = true;
    static constexpr bool PERSISTENT = false;
    static constexpr bool PREFETCH = false;
    struct Params {
        const uint4 *q4;
        const float *hs;
        const float *mass;
        const CorrRec *corr;
        float *rho;
    };
    struct Rec {
        uint4 q;
        float m;
    };
    struct IState {
        uint4 q;
        float inv_h, A, B[3], acc;
    };
    __device__ static void init(IState &s, int i, bool valid, const Params &p) {
        s.q = valid ? p.q4[i] : make_uint4(0, 0, 0, 0);
        s.inv_h = 1.f / (valid ? p.hs[i] : 1.f);
        const float4 c = valid ? p.corr[i].c0 : make_float4(0.f, 0.f, 0.f, 0.f);
        s.A = c.x;
        s.B[0] = c.y; s.B[1] = c.z; s.B[2] = c.w;
        s.acc = valid ? p.mass[i] : 0.f;                 // self: x = 0, W(0) / (495/(32 pi h^3)) = 1
    }
    __device__ static void zero(IState &s) { s.acc = 0.f; }
    __device__ static void merge(IState &s, const IState &o) { s.acc += o.acc; }
    __device__ static Rec load(uint32_t e, size_t, const Params &p) {
        const uint32_t j = e & 0x3fffffffu;
        return Rec{__ldg(p.q4 + j), __ldg(p.mass + j)};
    }
    __device__ static void pair(IState &s, const Rec &r, uint32_t, size_t, bool, const Params &) {
        int dx = (int)(s.q.x - r.q.x), dy = (int)(s.q.y - r.q.y), dz = (int)(s.q.z - r.q.z);
        Sep d = separation(dx, dy, dz);
        float eta = d.r * s.inv_h;
        float t = fmaxf(1.f - eta, 0.f);
        float t2 = t * t, t3 = t2 * t;
        float Wu = t3 * t3 * fmaf(eta, fmaf(eta, K35_3, 6.f), 1.f);
        float sB = fmaf(s.B[0], d.x, fmaf(s.B[1], d.y, fmaf(s.B[2], d.z, 1.f)));
        s.acc = fmaf(r.m * sB, Wu, s.acc);
    }
    __device__ static void finish(IState &s, int i, const Params &p) {
        const float ih3 = s.inv_h * s.inv_h * s.inv_h;
        p.rho[i] = s.A * (KW * ih3) * s.acc;
    }
};

int run_density(crk_ctx *ctx, cudaStream_t s) {
    PD::Params p{ctx->q4, ctx->hs, ctx->mass, ctx->corr, ctx->rho};
    return launch_lpass<PD, 8>(ctx, PROF_DENS, p, s, "RK density");
}

int run_corrections(crk_ctx *ctx, bool with_gradv, cudaStream_t s) {
    int rc;
    if (ctx->p.precision == 3) {
        P2X::Params p{ctx->q4, ctx->qV, ctx->hs, ctx->corr};
        rc = launch_lpass<P2X, 4>(ctx, PROF_P2, p, s, "P2 corrections (float-float)");
    } else if (ctx->p.precision == 2) {
        typedef P2<true, true> K;
        K::Params p{ctx->q4, ctx->qV, ctx->hs, ctx->corr};
        rc = launch_lpass<K, 4>(ctx, PROF_P2, p, s, "P2 corrections");
    } else if (ctx->p.precision == 1) {
        typedef P2<true, false> K;
        K::Params p{ctx->q4, ctx->qV, ctx->hs, ctx->corr};
        rc = launch_lpass<K, 4>(ctx, PROF_P2, p, s, "P2 corrections");
    } else {
        typedef P2<false, false> K;
        K::Params p{ctx->q4, ctx->qV, ctx->hs, ctx->corr};
        rc = launch_lpass<K, 4>(ctx, PROF_P2, p, s, "P2 corrections");
    }
    if (rc || !with_gradv) return rc;
    if (ctx->p.precision >= 2) {
        P3<true>::Params p3{ctx->q4, ctx->qV, ctx->hs, ctx->vel, ctx->corr, ctx->gv, (float)(1.0 / ctx->p.a)};
        return launch_lpass<P3<true>, 4>(ctx, PROF_P3, p3, s, "P3 grad v");
    }
    P3<false>::Params p3{ctx->q4, ctx->qV, ctx->hs, ctx->vel, ctx->corr, ctx->gv, (float)(1.0 / ctx->p.a)};
    return launch_lpass<P3<false>, 4>(ctx, PROF_P3, p3, s, "P3 grad v");
}

}  // namespace crk
