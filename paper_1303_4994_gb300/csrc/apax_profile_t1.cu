// apax_profile_t1.cu -- the profiler sweep (Sec. 4) of float32 arrays with
// one codec block per thread.
//
// The sweep of Sec. 4 encodes the array at every candidate setting and
// compares the decoded y with x.  Here each thread owns one block of at most
// 256 samples and walks it a few times:
//   1. the block maximum (float block exponent Eb, Sec. 6 float header);
//   2. code 0: the three streams' packet sizes (the best-stream decision of
//      Sec. 6, shared with the next block's thread), candidate 0 and the
//      block sums of x;
//   3. the other candidates, five per walk, on the stream the predecessor
//      block chose (codes with k >= 24 need no walk: they quantise every
//      sample of a float32 block to 0; a lone last candidate, when the
//      walked codes number 1 more than a multiple of five, rides along in
//      step 2 on all three streams instead of taking a walk of its own).
// Nothing is exchanged between threads inside a walk (no team scans): the
// greedy JEE token count runs sequentially, three candidates at a time in
// 10-bit lanes of one register.
//
// Exact sums.  With X = x 2^(23-Eb), q0 = RNE(X) and the remainder
// R0 = (X - q0) 2^24 (an integer whenever |X| >= 1/2), and at candidate
// code 128k (a power-of-two attenuation 2^-k) y = q 2^(Eb-23+k):
//   sum y    = 2^(Eb-23+k) S,                    S = sum q
//   sum y^2  = 2^(2(Eb-23+k)) C,                 C = sum q^2
//   sum xy   = 2^(2(Eb-23)+k-24) (2^24 A + B),   A = sum q0 q, B = sum R0 q
//   A        = 2^k C + E,                        E = sum (q0 - 2^k q) q
//   sum d^2  = 2^(2Eb-94) (Sxx - 2^(k+49) A - 2^(k+25) B + 2^(2k+48) C)
//   sum x^2  = 2^(2Eb-94) Sxx,  Sxx = 2^48 sum q0^2 + 2^25 sum q0 R0 + sum R0^2
// E's terms are small: |q0 - 2^k q| <= 2^(k-1) (both round X, at steps 1
// and 2^k) and |q| <= 2^(23-k), so |(q0 - 2^k q) q| <= 2^22 and E over a
// block of at most 256 samples is a 32-bit sum; only B and C need 64 bits.
// q0 and R0 are recomputed per walk from x; every candidate sample then
// costs one FMA (quantiser), two integer multiply-adds (derivative), the
// width term, a shift and three integer multiply-adds (sums), two of them
// 64-bit.  Each block sum is
// rounded once to binary64 and the run's partial adds its 16 block values in
// block order, as the team kernel does, so the results are identical.
//
// Samples below 2^(Eb-24) quantise to 0 at every candidate: they enter only
// sum x, sum x^2 and sum d^2 (= their x^2), which take them from exact
// 256-bit side sums; their remainder is left out of the fixed-point sums.
// A ragged last block is padded with copies of its last sample (the
// last-group padding of Sec. 6 packets) and the copies' contributions are
// taken back out of the sums.  Blocks this path still does not cover --
// exponents outside [-80, 127 - kmax], non-finite values, samples deeper
// than the side grid, or a predecessor whose code-0 decision needs the exact
// path -- mark their run; the team kernel then sweeps the marked runs
// (k_profile_fix).
#include "apax_team.cuh"
#include "apax_exact.cuh"
#include "apax_kernels.h"

namespace apax {

namespace {

constexpr int kP = 64;   // threads per CTA = blocks per CTA (4 runs of 16)
constexpr int kC = 5;    // candidates per walk
constexpr float kMagic = 12582912.0f;  // 1.5 2^23
constexpr int kMagicBits = 0x4B400000;

// Three greedy JEE nibble counters (Sec. 6 token rules) in 10-bit lanes:
// per group g >= 1 with d = e_g - e_(g-1): a diff in [-1, 1] pairs with a
// pending one (0 nibbles) or opens a token (1); otherwise a diff in [-2, 2]
// costs 1 and anything else an absolute token of 2.  The first exponent is
// absolute (2 nibbles).
struct Jee3 {
    static constexpr uint32_t L1 = 0x00100401u, L2 = 0x00200802u, L3 = 0x00300C03u,
                              B9 = 0x20080200u;
    uint32_t nib, st, el;
    __device__ __forceinline__ void first(uint32_t E)
    {
        nib = L2;
        st = 0;
        el = E;
    }
    __device__ __forceinline__ void push(uint32_t E)
    {
        const uint32_t D = E + B9 - el;  // 512 + d per lane (|d| <= 32)
        const uint32_t sm = (((D + L1) & ~(D - L2)) & B9) >> 9;  // |d| <= 1
        const uint32_t s2 = (((D + L2) & ~(D - L3)) & B9) >> 9;  // |d| <= 2
        nib = nib + L2 - s2 - (sm & st);
        st = sm & ~st;
        el = E;
    }
    __device__ __forceinline__ int lane(int i) const { return (int)((nib >> (10 * i)) & 1023u); }
};

__device__ __forceinline__ uint32_t btw(uint32_t u) { return u ^ (u << 1); }
__device__ __forceinline__ uint32_t ewidth(uint32_t o) { return 32u - (uint32_t)__clz(o); }

__device__ __forceinline__ double pow2d(int e)  // 2^e, -1022 <= e <= 1023
{
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Correctly rounded binary64 of V 2^e (the scaling stays in binary64's
// normal range here, so it is exact after the integer's own rounding).
__device__ __forceinline__ double round_scaled(i128 V, int e)
{
    const int64_t lo = (int64_t)V;
    if ((i128)lo == V) return __dmul_rn(__ll2double_rn(lo), pow2d(e));
    return round_i128(V, e);
}

// This thread's block: groups [0, Gt), the last one holding nl samples
// (1..4; the rest are copies of the block's last sample).
struct Blk {
    const uint4 *xp;
    int Gt, nl;
    __device__ __forceinline__ uint4 group(int g) const
    {
        if (g == Gt - 1 && nl < 4) {
            const uint32_t *p = reinterpret_cast<const uint32_t *>(xp + g);
            uint32_t v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = __ldg(p + (i < nl ? i : nl - 1));
            return make_uint4(v[0], v[1], v[2], v[3]);
        }
        return __ldg(xp + g);
    }
    __device__ __forceinline__ uint32_t last() const
    {
        return __ldg(reinterpret_cast<const uint32_t *>(xp + (Gt - 1)) + (nl - 1));
    }
};

// A candidate's four block sums from its exact integer sums (attenuation
// 2^-k, k >= 1): v = {sum y, sum xy, sum y^2, sum d^2}, each rounded once.
__device__ __forceinline__ void cand_sums(int k, int Eb, int S, int64_t Cs, int Es, int64_t Bs,
                                          const i128 &Sxx, bool tiny, const uint64_t *txx,
                                          double *v, int stride)
{
    const int64_t Ac = (Cs << k) + (int64_t)Es;  // sum q0 q
    const int sy = Eb - 23 + k;
    v[0] = __dmul_rn((double)S, pow2d(sy));
    v[stride] = round_scaled(((i128)Ac << 24) + (i128)Bs, 2 * (Eb - 23) + k - 24);
    v[2 * stride] = __dmul_rn(__ll2double_rn(Cs), pow2d(2 * sy));
    const i128 D = Sxx - ((i128)Ac << (k + 49)) - ((i128)Bs << (k + 25)) + ((i128)Cs << (2 * k + 48));
    if (tiny) {
        // D >= 0: sum (X - y)^2 of the other samples, in units of 2^-48
        W256 w;
#pragma unroll
        for (int i = 0; i < 4; ++i) w.l[i] = txx[i];
        w256_add(w, (u128)D, 145, false);
        v[3 * stride] = round_w256(w, 2 * Eb - 239);
    } else {
        v[3 * stride] = round_scaled(D, 2 * Eb - 94);
    }
}

// One walk over the block for M candidates (codes[0 .. M)), all k >= 1.
// Writes the candidates' four block sums to sv[4c + q][t] and their packet
// bytes; txx (tiny blocks) is the side sum of the tiny samples' x^2 on the
// grid 2^(2Eb - 239).
template <int M>
__device__ __forceinline__ void walk(const Blk &B, int Eb, int s, const uint32_t *codes, float b0,
                                     float b24, i128 Sxx, bool tiny, const uint64_t *txx,
                                     double (*sv)[kP], int t, uint32_t (&bytes)[kC])
{
    float bk[M];
    uint32_t qp[M], qpp[M];
    int S[M], se[M], Es[M];
    uint32_t kk[M];
    int64_t Cs[M], Bs[M];
    Jee3 jj[(M + 2) / 3];
    const uint32_t ca = s == 0 ? 0u : (s == 1 ? 1u : 2u), cb = s == 2 ? 1u : 0u;
    const float x0 = __uint_as_float(__ldg(reinterpret_cast<const uint32_t *>(B.xp)));
#pragma unroll
    for (int c = 0; c < M; ++c) {
        const int k = (int)(codes[c] >> 7);
        bk[c] = __int_as_float((150 - Eb - k) << 23);  // 2^(23 - Eb - k)
        const uint32_t qf = (uint32_t)(__float_as_int(__fmaf_rn(x0, bk[c], kMagic)) - kMagicBits);
        qp[c] = s == 2 ? qf : 0u;  // S1 starts from 0, S2 from q_0 (u_0 = q_0, u_1 = q_1 - q_0)
        qpp[c] = 2u * qf;
        S[c] = 0;
        se[c] = 0;
        kk[c] = (uint32_t)k;
        Es[c] = 0;
        Cs[c] = Bs[c] = 0;
    }
    uint4 vn = B.group(0);  // the next group's samples are loaded one iteration ahead
#pragma unroll 1
    for (int g = 0; g < B.Gt; ++g) {
        const uint4 v = vn;
        if (g + 1 < B.Gt) vn = B.group(g + 1);
        const float xf[4] = {__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                             __uint_as_float(v.w)};
        int q0[4], R0[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            q0[i] = __float2int_rn(__fmul_rn(xf[i], b0));
            R0[i] = __float2int_rn(__fmaf_rn(__int2float_rn(q0[i]), -16777216.0f, __fmul_rn(xf[i], b24)));
        }
        uint32_t ev[M];
#pragma unroll
        for (int c = 0; c < M; ++c) {
            uint32_t o = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = __float_as_int(__fmaf_rn(xf[i], bk[c], kMagic)) - kMagicBits;
                const uint32_t u = (uint32_t)q - ca * qp[c] + cb * qpp[c];
                o |= btw(u);
                qpp[c] = qp[c];
                qp[c] = (uint32_t)q;
                S[c] += q;
                Cs[c] += (int64_t)q * q;
                // sum q0 q = 2^k sum q^2 + sum e q, e = q0 - 2^k q, |e q| <= 2^22
                // (a tiny sample has q0 = q = 0 and its R0 adds nothing)
                Es[c] += (q0[i] - (int)((uint32_t)q << kk[c])) * q;
                Bs[c] += (int64_t)R0[i] * q;
            }
            ev[c] = ewidth(o);
            se[c] += (int)ev[c];
        }
#pragma unroll
        for (int t3 = 0; t3 < (M + 2) / 3; ++t3) {
            uint32_t E = ev[3 * t3];
            if (3 * t3 + 1 < M) E |= ev[3 * t3 + 1] << 10;
            if (3 * t3 + 2 < M) E |= ev[3 * t3 + 2] << 20;
            if (g == 0) jj[t3].first(E);
            else jj[t3].push(E);
        }
    }
    // a ragged block: take the padding copies of its last sample back out
    const int pad = 4 - B.nl;
    int pq0 = 0, pR0 = 0;
    float pxf = 0.f;
    if (pad) {
        pxf = __uint_as_float(B.last());
        pq0 = __float2int_rn(__fmul_rn(pxf, b0));
        pR0 = __float2int_rn(__fmaf_rn(__int2float_rn(pq0), -16777216.0f, __fmul_rn(pxf, b24)));
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
        const int k = (int)(codes[c] >> 7);
        if (pad) {
            const int q = __float_as_int(__fmaf_rn(pxf, bk[c], kMagic)) - kMagicBits;
            S[c] -= pad * q;
            Cs[c] -= (int64_t)pad * ((int64_t)q * q);
            Es[c] -= pad * ((pq0 - (int)((uint32_t)q << kk[c])) * q);
            Bs[c] -= (int64_t)pad * ((int64_t)pR0 * q);
        }
        const int nib = jj[c / 3].lane(c % 3);
        const uint32_t bits = 48u + 4u * (uint32_t)nib + 4u * (uint32_t)se[c];
        bytes[c] = 4u * ((bits + 31u) >> 5);
        cand_sums(k, Eb, S[c], Cs[c], Es[c], Bs[c], Sxx, tiny, txx, &sv[4 * c][t], kP);
    }
}

template <int M>
__device__ __forceinline__ void walk_dispatch(int m, const Blk &B, int Eb, int s,
                                              const uint32_t *codes, float b0, float b24, i128 Sxx,
                                              bool tiny, const uint64_t *txx, double (*sv)[kP],
                                              int t, uint32_t (&bytes)[kC])
{
    if constexpr (M >= 1) {
        if (m == M) walk<M>(B, Eb, s, codes, b0, b24, Sxx, tiny, txx, sv, t, bytes);
        else walk_dispatch<M - 1>(m, B, Eb, s, codes, b0, b24, Sxx, tiny, txx, sv, t, bytes);
    }
}

// The run partials of one group of quantities: run r of the CTA adds the
// values of its active blocks in block order (from 0.0, like the team
// kernel) and writes run_sums[run][q0 + i].
__device__ __forceinline__ void run_partials(const ProfArgs &a, double (*sv)[kP], int nq, int q0,
                                             uint64_t jfirst)
{
    const int Qn = 2 + 4 * a.ncand;
    for (int w = threadIdx.x; w < 4 * nq; w += kP) {
        const int r = w / nq, i = w % nq;
        const uint64_t jb = jfirst + 16ull * (uint64_t)r;
        if (jb >= a.nb || jb >= a.run1 * 16ull) continue;
        double acc = 0.0;
#pragma unroll 4
        for (int b = 0; b < 16; ++b)
            if (jb + (uint64_t)b < a.nb) acc = __dadd_rn(acc, sv[i][16 * r + b]);
        a.run_sums[(jb / 16) * (uint64_t)Qn + (uint64_t)(q0 + i)] = acc;
    }
}

// The code-0 pass (one block, one thread): the three streams' packet bits
// at code 0 (the best-stream decision), candidate 0's sums and the block's
// sums of x; with LONE, also one more candidate (code 128 kL) on all three
// streams.  R0 is zeroed for tiny samples (their x enters through the side
// sums); their q0 and q are 0 at every code.
struct Code0 {
    uint32_t bits3[3] = {0u, 0u, 0u};
    int64_t Sq0 = 0, SR0 = 0, C0 = 0, A0 = 0, B0 = 0;
    bool tiny = false;
    int kL = 1;
    uint32_t bitsL[3] = {0u, 0u, 0u};
    int SL = 0, EL = 0;
    int64_t CL = 0, BL = 0;
};

template <bool LONE>
__device__ __forceinline__ void code0_pass(const Blk &B, float b0, float b24, uint32_t tthr, int eb,
                                           Code0 &z)
{
    const float x0 = __uint_as_float(__ldg(reinterpret_cast<const uint32_t *>(B.xp)));
    const int qf = __float2int_rn(__fmul_rn(x0, b0));
    uint32_t qp1 = 0, qp2 = (uint32_t)qf, qpp2 = 2u * (uint32_t)qf;
    Jee3 j3;
    int se0 = 0, se1 = 0, se2 = 0;
    // the lone candidate: 2^(23 - Eb - kL) (clamped: blocks out of range
    // are swept again by the team kernel)
    const float bkL = __int_as_float(min(max(150 - eb - z.kL, 1), 254) << 23);
    const uint32_t kL = (uint32_t)z.kL;
    const int qfL = LONE ? __float_as_int(__fmaf_rn(x0, bkL, kMagic)) - kMagicBits : 0;
    uint32_t lp1 = 0, lp2 = (uint32_t)qfL, lpp2 = 2u * (uint32_t)qfL;
    Jee3 jL;
    int sL0 = 0, sL1 = 0, sL2 = 0;
    int SL = 0, EL = 0;
    int64_t CL = 0, BL = 0;
    int64_t Sq0 = 0, SR0 = 0, C0 = 0, A0 = 0, B0 = 0;
    bool tiny = false;
    // the next two groups are loaded ahead (the block's first per-thread
    // read after the coalesced maximum: mostly from L2)
    uint4 vn1 = B.group(0), vn2 = B.Gt > 1 ? B.group(1) : vn1;
#pragma unroll 1
    for (int g = 0; g < B.Gt; ++g) {
        const uint4 v = vn1;
        vn1 = vn2;
        if (g + 2 < B.Gt) vn2 = B.group(g + 2);
        const uint32_t xv[4] = {v.x, v.y, v.z, v.w};
        uint32_t o0 = 0, o1 = 0, o2 = 0, l0 = 0, l1 = 0, l2 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float xf = __uint_as_float(xv[i]);
            const bool ti = ((xv[i] & 0x7fffffffu) - 1u) < tthr - 1u;
            tiny |= ti;
            const int q = __float2int_rn(__fmul_rn(xf, b0));
            int R = __float2int_rn(__fmaf_rn(__int2float_rn(q), -16777216.0f, __fmul_rn(xf, b24)));
            R = ti ? 0 : R;  // a tiny sample's x enters through the side sums
            const uint32_t uq = (uint32_t)q;
            o0 |= btw(uq);
            o1 |= btw(uq - qp1);
            o2 |= btw(uq - 2u * qp2 + qpp2);
            qp1 = uq;
            qpp2 = qp2;
            qp2 = uq;
            Sq0 += q;
            SR0 += R;
            C0 += (int64_t)q * q;
            A0 += (int64_t)q * R;
            B0 += (int64_t)R * R;
            if constexpr (LONE) {
                const int ql = __float_as_int(__fmaf_rn(xf, bkL, kMagic)) - kMagicBits;
                const uint32_t ul = (uint32_t)ql;
                l0 |= btw(ul);
                l1 |= btw(ul - lp1);
                l2 |= btw(ul - 2u * lp2 + lpp2);
                lp1 = ul;
                lpp2 = lp2;
                lp2 = ul;
                SL += ql;
                CL += (int64_t)ql * ql;
                EL += (q - (int)(ul << kL)) * ql;  // |(q0 - 2^k q) q| <= 2^22
                BL += (int64_t)R * ql;             // (R = 0 where q = 0)
            }
        }
        const uint32_t e0 = ewidth(o0), e1 = ewidth(o1), e2 = ewidth(o2);
        se0 += (int)e0;
        se1 += (int)e1;
        se2 += (int)e2;
        const uint32_t E = e0 | (e1 << 10) | (e2 << 20);
        if (g == 0) j3.first(E);
        else j3.push(E);
        if constexpr (LONE) {
            const uint32_t f0 = ewidth(l0), f1 = ewidth(l1), f2 = ewidth(l2);
            sL0 += (int)f0;
            sL1 += (int)f1;
            sL2 += (int)f2;
            const uint32_t F = f0 | (f1 << 10) | (f2 << 20);
            if (g == 0) jL.first(F);
            else jL.push(F);
        }
    }
    z.bits3[0] = 48u + 4u * (uint32_t)(j3.lane(0) + se0);
    z.bits3[1] = 48u + 4u * (uint32_t)(j3.lane(1) + se1);
    z.bits3[2] = 48u + 4u * (uint32_t)(j3.lane(2) + se2);
    // the padding copies of a ragged block's last sample
    const int pad = 4 - B.nl;
    if (pad) {
        const uint32_t xl = B.last();
        const float xf = __uint_as_float(xl);
        const bool ti = ((xl & 0x7fffffffu) - 1u) < tthr - 1u;
        const int q = __float2int_rn(__fmul_rn(xf, b0));
        int R = __float2int_rn(__fmaf_rn(__int2float_rn(q), -16777216.0f, __fmul_rn(xf, b24)));
        R = ti ? 0 : R;
        Sq0 -= pad * q;
        SR0 -= pad * R;
        C0 -= (int64_t)pad * ((int64_t)q * q);
        A0 -= (int64_t)pad * ((int64_t)q * R);
        B0 -= (int64_t)pad * ((int64_t)R * R);
        if constexpr (LONE) {
            const int ql = __float_as_int(__fmaf_rn(xf, bkL, kMagic)) - kMagicBits;
            SL -= pad * ql;
            CL -= (int64_t)pad * ((int64_t)ql * ql);
            EL -= pad * ((q - (int)((uint32_t)ql << kL)) * ql);
            BL -= (int64_t)pad * ((int64_t)R * ql);
        }
    }
    z.Sq0 = Sq0;
    z.SR0 = SR0;
    z.C0 = C0;
    z.A0 = A0;
    z.B0 = B0;
    z.tiny = tiny;
    if constexpr (LONE) {
        z.bitsL[0] = 48u + 4u * (uint32_t)(jL.lane(0) + sL0);
        z.bitsL[1] = 48u + 4u * (uint32_t)(jL.lane(1) + sL1);
        z.bitsL[2] = 48u + 4u * (uint32_t)(jL.lane(2) + sL2);
        z.SL = SL;
        z.EL = EL;
        z.CL = CL;
        z.BL = BL;
    }
}

// 8 CTAs of 64 threads per SM (at most 128 registers): 1216 resident warps
// take the 2048 warps of a 64 MiB float32 array in one wave with room to spare.
__global__ void __launch_bounds__(kP, 8) k_profile_f32_t1(ProfArgs a)
{
    __shared__ double s_v[4 * kC][kP];
    __shared__ double s_lone[4][kP];
    __shared__ uint32_t s_lone_b[kP];
    __shared__ uint64_t s_txx[kP][4];
    __shared__ int s_best[kP / 32];
    __shared__ int s_halo;
    __shared__ uint32_t s_codes[32];
    if (threadIdx.x < 32) s_codes[threadIdx.x] = threadIdx.x < a.ncand ? a.codes[threadIdx.x] : 0u;

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint64_t jfirst = a.run0 * 16ull + (uint64_t)blockIdx.x * kP;
    const uint64_t jend = a.run1 * 16ull < a.nb ? a.run1 * 16ull : a.nb;
    const uint64_t j = jfirst + (uint64_t)t;
    const bool active = j < jend;
    const uint32_t N = a.N;
    const int G = (int)(N >> 2);
    Blk B;
    B.xp = reinterpret_cast<const uint4 *>(a.x) + (active ? j * (uint64_t)G : 0);
    {
        const uint64_t L = active ? (a.n - j * (uint64_t)N < N ? a.n - j * (uint64_t)N : N) : 0;
        B.Gt = (int)((L + 3) >> 2);
        B.nl = (int)(L - 4 * (uint64_t)(B.Gt ? B.Gt - 1 : 0));
        if (!active) B.nl = 4;
    }
    int kmax = 0;
    for (int c = 1; c < a.ncand; ++c) kmax = max(kmax, (int)(a.codes[c] >> 7));  // (param space)

    // the decision of block jfirst - 1 (code 0, three streams), teams of 32
    if (wid == 0) {
        int hb = -1;
        if (jfirst > 0 && jfirst < jend) {
            TBlock<4> pv;
            open_team_block<4, 32>(pv, reinterpret_cast<const float *>(a.x), a.n, N, a.nb, jfirst - 1,
                                   (G + 31) / 32);
            hb = team_best_stream<4, 32>(pv, false);  // version-1 byte counts only
        }
        if (lane == 0) s_halo = hb;
    }

    // ---- 1. block maximum.  When the warp's 32 blocks are whole and a block
    // is a multiple of 32 groups, the warp reads them together (coalesced:
    // lane l takes group 32i + l of a block) and reduces each block with one
    // REDUX; the first read of the array from DRAM is then contiguous.
    uint32_t mx = 0;
    const bool whole = (j + 1) * (uint64_t)N <= a.n && j < jend;
    if (__all_sync(kFull, whole) && (G & 31) == 0) {
        // four blocks per step, their loads issued together (the reads come
        // from DRAM; one block at a time left a load's latency per block)
        const uint4 *wb = reinterpret_cast<const uint4 *>(a.x) + (j - (uint64_t)lane) * (uint64_t)G;
#pragma unroll 1
        for (int b = 0; b < 32; b += 4) {
            uint32_t lm[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
            for (int i = 0; i < (G >> 5); i += 2) {
                uint4 v[4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        v[u][h] = i + h < (G >> 5) ? __ldg(wb + (uint64_t)(b + u) * G + 32 * (i + h) + lane)
                                                   : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        lm[u] = max(lm[u], max(max(v[u][h].x & 0x7fffffffu, v[u][h].y & 0x7fffffffu),
                                               max(v[u][h].z & 0x7fffffffu, v[u][h].w & 0x7fffffffu)));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t r = __reduce_max_sync(kFull, lm[u]);
                if (lane == b + u) mx = r;
            }
        }
    } else {
#pragma unroll 4
        for (int g = 0; g < B.Gt; ++g) {
            const uint4 v = B.group(g);
            mx = max(mx, max(max(v.x & 0x7fffffffu, v.y & 0x7fffffffu),
                             max(v.z & 0x7fffffffu, v.w & 0x7fffffffu)));
        }
    }
    const bool bad = mx >= 0x7f800000u;
    const int Eb = (active && !bad) ? block_exp_from_maxbits<4>((uint64_t)mx) : 0;
    // exact code-0 decision: the scale 2^(23 - Eb) is a normal float
    const bool dv = active && !bad && Eb >= -100;
    bool fb = active && (bad || Eb < -80 || Eb + kmax > 127);

    // ---- 2. code 0: three streams, candidate 0, block sums
    const int eb = dv ? Eb : 0;
    const float b0 = __int_as_float((150 - eb) << 23);                   // 2^(23 - Eb)
    const float b24 = __int_as_float(min(max(174 - eb, 1), 254) << 23);  // 2^(47 - Eb)
    const uint32_t tthr = (uint32_t)max(eb + 103, 1) << 23;              // |x| < 2^(Eb-24)
    // the walks' lone last candidate: when the walked codes number 1 more
    // than a multiple of kC, the last one is taken in the code-0 pass (on
    // all three streams: the block's stream is known only after it) instead
    // of in a walk of its own
    int ct = a.ncand;
    while (ct > 1 && (a.codes[ct - 1] >> 7) >= 24) --ct;
    const bool lone = ct > 1 && (ct - 1) % kC == 1;
    Code0 z;
    z.kL = lone ? (int)(a.codes[ct - 1] >> 7) : 1;
    if (dv) {
        if (lone) code0_pass<true>(B, b0, b24, tthr, eb, z);
        else code0_pass<false>(B, b0, b24, tthr, eb, z);
    }
    const uint32_t bits3[3] = {z.bits3[0], z.bits3[1], z.bits3[2]};
    const int64_t Sq0 = z.Sq0, SR0 = z.SR0, C0 = z.C0, A0 = z.A0, B0 = z.B0;
    const bool tiny = z.tiny;
    // tiny samples (0 < |x| < 2^(Eb-24)): exact side sums of x on the grid
    // 2^(Eb-237) and of x^2 on 2^(2Eb-239); deeper ones go to the team path
    W256 tx, txx;
    w256_zero(tx);
    w256_zero(txx);
    if (tiny) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(B.xp);
        const int L = 4 * (B.Gt - 1) + B.nl;
        for (int i = 0; i < L; ++i) {
            const uint32_t v = __ldg(p + i);
            if (((v & 0x7fffffffu) - 1u) >= tthr - 1u) continue;
            const int bexp = (int)((v >> 23) & 0xff);
            const int ex = (bexp ? bexp : 1) - 150;
            const uint32_t Mt = (v & 0x7fffffu) | (bexp ? 0x800000u : 0u);
            const int px = ex - (Eb - 237), pxx = 2 * ex - (2 * Eb - 239);
            if (px < 0 || pxx < 0) {
                fb = true;
                continue;
            }
            w256_add(tx, (u128)Mt, px, (v >> 31) != 0);
            w256_add(txx, (u128)((uint64_t)Mt * Mt), pxx, false);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) s_txx[t][i] = txx.l[i];
    int best = 0;
    if (bits3[1] < bits3[best]) best = 1;
    if (bits3[2] < bits3[best]) best = 2;
    // stream of block j = best(j - 1): neighbour lane, previous warp, or the halo
    int pbest = __shfl_up_sync(kFull, best, 1);
    int pdv = __shfl_up_sync(kFull, (int)dv, 1);
    if (lane == 31) s_best[wid] = best | ((int)dv << 2);
    __syncthreads();
    if (lane == 0) {
        if (wid > 0) {
            pbest = s_best[wid - 1] & 3;
            pdv = s_best[wid - 1] >> 2;
        } else {
            pbest = s_halo;
            pdv = 1;  // the halo decision is exact (team path)
        }
    }
    const int s = j == 0 ? best : pbest;
    if (active && j > 0 && !pdv) fb = true;
    // a run goes to the exact team path if any of its blocks does
    const unsigned fbm = __ballot_sync(kFull, fb);
    const bool runfb = ((fbm >> (lane & 16)) & 0xffffu) != 0;
    if ((lane & 15) == 0 && active) a.run_flags[j / 16] = runfb ? 1 : 0;
    const bool go = active && !runfb;

    // candidate 0 and the block sums
    const i128 Sxx = ((i128)C0 << 48) + ((i128)A0 << 25) + (i128)B0;
    double sxx_blk = 0.0;  // the block's sum x^2, rounded once
    {
        double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (go) {
            const int64_t X24 = (Sq0 << 24) + SR0;  // sum X 2^24 of the other samples
            if (tiny) {
                W256 w = tx;
                w256_add(w, (u128)(X24 < 0 ? -X24 : X24), 190, X24 < 0);
                v[0] = round_w256(w, Eb - 237);
                w = txx;
                w256_add(w, (u128)Sxx, 145, false);
                v[1] = round_w256(w, 2 * Eb - 239);
                w = txx;
                w256_add(w, (u128)B0, 145, false);
                v[5] = round_w256(w, 2 * Eb - 239);
            } else {
                v[0] = __dmul_rn(__ll2double_rn(X24), pow2d(Eb - 47));
                v[1] = round_scaled(Sxx, 2 * Eb - 94);
                v[5] = __dmul_rn(__ll2double_rn(B0), pow2d(2 * Eb - 94));
            }
            v[2] = __dmul_rn(__ll2double_rn(Sq0), pow2d(Eb - 23));
            v[3] = round_scaled(((i128)C0 << 24) + (i128)A0, 2 * (Eb - 23) - 24);
            v[4] = __dmul_rn(__ll2double_rn(C0), pow2d(2 * (Eb - 23)));
        }
        sxx_blk = v[1];
#pragma unroll
        for (int i = 0; i < 6; ++i) s_v[i][t] = v[i];
        const uint32_t bs = s == 0 ? bits3[0] : (s == 1 ? bits3[1] : bits3[2]);
        uint32_t by = go ? 4u * ((bs + 31u) >> 5) : 0u;
#pragma unroll
        for (int m = 8; m >= 1; m >>= 1) by += __shfl_xor_sync(kFull, by, m);
        if ((lane & 15) == 0 && go) atomicAdd(a.bytes + 0, (unsigned long long)by);
    }
    // the lone candidate's sums and bytes, parked until its turn in step 3
    if (lone) {
        double lv[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t lb = 0u;
        if (go) {
            cand_sums(z.kL, Eb, z.SL, z.CL, z.EL, z.BL, Sxx, tiny, txx.l, lv, 1);
            const uint32_t bl = s == 0 ? z.bitsL[0] : (s == 1 ? z.bitsL[1] : z.bitsL[2]);
            lb = 4u * ((bl + 31u) >> 5);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) s_lone[i][t] = lv[i];
        s_lone_b[t] = lb;
    }
    __syncthreads();
    run_partials(a, s_v, 6, 0, jfirst);
    __syncthreads();

    // ---- 3. the other candidates, kC per walk.  An attenuation 2^-k with
    // k >= 24 quantises every sample to 0 (|X| < 2^23, so |X 2^-k| < 1/2):
    // such a candidate's sums of y, xy and y^2 are 0, its sum d^2 is the
    // block's sum x^2, and its packet has every exponent 0 (the first one
    // absolute, the rest zero diffs, two to a joint token), so it takes no
    // walk.  The codes increase, so these candidates end the list.
    // (ct: the first such code, from step 2)
    const uint32_t zero_bytes = 4u * ((48u + 4u * (uint32_t)(2 + B.Gt / 2) + 31u) >> 5);
    for (int c0 = 1; c0 < a.ncand;) {
        const bool trivial = c0 >= ct;
        const bool folded = lone && c0 == ct - 1;  // the lone candidate, from step 2
        const int m = folded ? 1 : min(kC, (trivial ? a.ncand : ct) - c0);
        uint32_t bytes[kC];
#pragma unroll
        for (int i = 0; i < kC; ++i) bytes[i] = 0u;
        if (go && folded) {
#pragma unroll
            for (int i = 0; i < 4; ++i) s_v[i][t] = s_lone[i][t];
            bytes[0] = s_lone_b[t];
        } else if (go && !trivial) {
            walk_dispatch<kC>(m, B, Eb, s, s_codes + c0, b0, b24, Sxx, tiny, s_txx[t], s_v, t, bytes);
        } else if (go) {
#pragma unroll
            for (int i = 0; i < kC; ++i) {
                if (i < m) {
                    s_v[4 * i + 0][t] = 0.0;
                    s_v[4 * i + 1][t] = 0.0;
                    s_v[4 * i + 2][t] = 0.0;
                    s_v[4 * i + 3][t] = sxx_blk;
                    bytes[i] = zero_bytes;
                }
            }
        } else {
            for (int i = 0; i < 4 * m; ++i) s_v[i][t] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            if (c >= m) break;
            uint32_t by = bytes[c];
#pragma unroll
            for (int w = 8; w >= 1; w >>= 1) by += __shfl_xor_sync(kFull, by, w);
            if ((lane & 15) == 0 && go) atomicAdd(a.bytes + c0 + c, (unsigned long long)by);
        }
        __syncthreads();
        run_partials(a, s_v, 4 * m, 2 + 4 * c0, jfirst);
        __syncthreads();
        c0 += m;
    }
}

}  // namespace

bool profile_t1_eligible(const ProfArgs &a)
{
    if (a.dtype != 4 || !a.run_flags || a.N > 256 || a.ncand < 1 || a.codes[0] != 0) return false;
    if (a.gsh || a.sum) return false;  // version-1 byte counts only
    if (((uintptr_t)a.x & 15) || a.nb < kProfT1MinBlocks) return false;
    for (int c = 1; c < a.ncand; ++c) {
        const uint32_t code = a.codes[c];
        if ((code & 127) || code < 128 || code > 3968) return false;
    }
    return true;
}

cudaError_t launch_profile_t1(const ProfArgs &a, cudaStream_t s)
{
    const uint64_t blocks = (a.run1 - a.run0) * 16;
    const uint64_t grid = (blocks + kP - 1) / kP;
    if (grid) k_profile_f32_t1<<<(unsigned)grid, kP, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace apax
