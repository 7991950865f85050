// apax_profile.cu -- profiler sweep (Sec. 4): for every candidate code, the
// exact fixed-quality packet sizes and the reconstruction sums of the decoded
// y against x, in one pass that reads the input once.
//
// A team of 8 threads owns one block; a CTA's 16 teams are one run of 16
// consecutive blocks (a level-1 node of the fan-in-16 summation tree).  Per
// block: the stream decision (the predecessor at code 0, one-block lag of
// Sec. 6), then per candidate the chosen stream's exponents and JEE token
// count (packet size) and the exact block sums.
//
// Candidates are any increasing codes.  For the power-of-two attenuations
// a = 2^-k (codes with m = 0) and floats the decoded value is exactly
// y = q 2^s with s = Eb - Q + k, so with the quantiser remainder
// d = x - y = D' 2^(s-P):
//   sum y    = 2^s  sum q
//   sum y^2  = 2^2s A,               A = sum q^2
//   sum xy   = 2^2s A + 2^(2s-P) B,  B = sum q D'
//   sum d^2  = sum x^2 - 2^2s A - 2^(2s-P+1) B
// all exact in 64/128/256-bit integers.  Blocks with values too small for
// the fixed-point window of sum x^2, candidates whose y leaves the normal
// range, and float candidates with m != 0 (y = q R[m] 2^(s-24) rounded to
// the format, the decoder's reciprocal table) take an exact fallback with a
// shared-memory superaccumulator.  Integer candidates dequantise with the
// decoder's formula directly.  Each
// block sum is rounded once to binary64 and added into the run's partial in
// block order.
#include <type_traits>

#include "apax_team.cuh"
#include "apax_exact.cuh"
#include "apax_kernels.h"
#include "apax_plan.h"

namespace apax {

namespace {

constexpr int TS = kProfTS;
static_assert(TS >= 8, "the exact fallback rounds its six sums on team threads 0..5");
constexpr int kRun = 16;   // blocks per CTA = one tree node
constexpr int kWin = 200;  // f64: window LSB = 2^(2 Eb - kWin) for sum x^2

__device__ __forceinline__ void set_status(int *st, int code) { atomicMin(st, code); }

__device__ __forceinline__ uint32_t shl_clamp(uint32_t v, int s)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"((uint32_t)s));  // 0 for s >= 32
    return r;
}

template <int DT>
struct FDec {
    uint64_t M;
    int ex;
    bool neg;
};

template <int DT>
__device__ __forceinline__ FDec<DT> fdec(typename LaneT<DT>::t v)
{
    using T = DT_<DT>;
    using B = typename T::bits;
    FDec<DT> d;
    const int bexp = (int)((v >> T::MB) & (B)T::EMAX);
    d.M = (uint64_t)(v & (((B)1 << T::MB) - 1)) | (bexp ? ((uint64_t)1 << T::MB) : 0);
    d.ex = (bexp ? bexp : 1) - T::BIAS - T::MB;
    d.neg = (v >> (sizeof(B) * 8 - 1)) & 1;
    return d;
}

// team reductions of wide integers (shuffles of 32-bit pieces)
__device__ __forceinline__ int64_t team_sum_i64(int64_t v)
{
#pragma unroll
    for (int m = TS / 2; m >= 1; m >>= 1) v += tshfl_xor<TS>(v, m);
    return v;
}
__device__ __forceinline__ i128 team_sum_i128(i128 v)
{
#pragma unroll
    for (int m = TS / 2; m >= 1; m >>= 1) {
        const uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
        const uint64_t olo = tshfl_xor<TS>(lo, m), ohi = tshfl_xor<TS>(hi, m);
        v += (i128)(((u128)ohi << 64) | olo);
    }
    return v;
}
__device__ __forceinline__ W256 team_sum_w256(W256 a)
{
#pragma unroll
    for (int m = TS / 2; m >= 1; m >>= 1) {
        W256 o;
#pragma unroll
        for (int i = 0; i < 4; ++i) o.l[i] = tshfl_xor<TS>(a.l[i], m);
        uint64_t carry = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t s1 = a.l[i] + o.l[i];
            const uint64_t c1 = s1 < a.l[i];
            const uint64_t s2 = s1 + carry;
            carry = c1 | (s2 < s1);
            a.l[i] = s2;
        }
    }
    return a;
}

// per (team, candidate) staging
// float: sum q, A, B; int: sum y, sum xy, sum y^2, sum d^2.  64-bit for
// float32, int8 and int16 (every per-block sum fits), 128-bit otherwise.
template <typename V>
struct CandStageT {
    V sq, A, B, D;
    uint32_t bits;
    int fast;
};
template <int DT>
using CandStage = CandStageT<typename std::conditional<DT == 5 || DT == 3, i128, int64_t>::type>;

template <int DT>
struct PS {
    static constexpr int ND = DT == 5 ? 144 : 26;     // superaccumulator digits
    static constexpr int LO = DT == 5 ? -2304 : -320;  // position of digit 0
};

// Exact fallback for the block sums (want_block: x, x^2) or one candidate
// (y, xy, y^2, d^2), by one team with shared-memory atomics.  acc: 6 ND
// digits.  The whole CTA calls it; only team `who` works.
template <int DT>
__device__ void fallback_team(const TBlock<DT> &b, int code, bool want_block,
                              bool want_cand, long long *accmem, double *dst_block,
                              double *dst_cand, bool me)
{
    using T = DT_<DT>;
    constexpr int ND = PS<DT>::ND, LO = PS<DT>::LO;
    const int t = tlane<TS>();
    const unsigned tm = ((1u << TS) - 1u) << (lane_id() & ~(unsigned)(TS - 1));
    if (me) {
        for (int i = t; i < 6 * ND; i += TS) accmem[i] = 0;
        __syncwarp(tm);
        SmemAcc<ND, LO> acc[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i].d = accmem + i * ND;
        const Quant<DT> Q(code, b.Eb);
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT>(b, 4 * g, xv);
            for (int k = 0; k < 4; ++k) {
                if (4 * g + k >= b.L) continue;
                const FDec<DT> dx = fdec<DT>(xv[k]);
                const u128 xx = (u128)dx.M * dx.M;
                if (want_block) {
                    acc[0].add(dx.M, dx.ex, dx.neg);
                    acc[2].add(xx, 2 * dx.ex, false);
                }
                if (want_cand) {
                    const int32_t q = Q(xv[k]);
                    typename T::bits yb =
                        q ? round_to_format<DT>((int64_t)q * (int64_t)recip_entry(code & 127),
                                                b.Eb - T::Q + (code >> 7) - 24)
                          : 0;
                    FDec<DT> dy = fdec<DT>(yb);
                    if (!q) dy.M = 0;
                    const u128 xy = (u128)dx.M * dy.M, yy = (u128)dy.M * dy.M;
                    acc[1].add(dy.M, dy.ex, dy.neg);
                    acc[3].add(xy, dx.ex + dy.ex, dx.neg != dy.neg);
                    acc[4].add(yy, 2 * dy.ex, false);
                    acc[5].add(xx, 2 * dx.ex, false);
                    acc[5].add(xy, dx.ex + dy.ex + 1, dx.neg == dy.neg);
                    acc[5].add(yy, 2 * dy.ex, false);
                }
            }
        }
        __syncwarp(tm);
        // threads round different accumulators: x, y, x^2, xy, y^2, d^2
        if (want_block && t == 0) dst_block[0] = acc[0].round_inplace();
        if (want_block && t == 2) dst_block[1] = acc[2].round_inplace();
        if (want_cand && t == 1) dst_cand[0] = acc[1].round_inplace();
        if (want_cand && t == 3) dst_cand[1] = acc[3].round_inplace();
        if (want_cand && t == 4) dst_cand[2] = acc[4].round_inplace();
        if (want_cand && t == 5) dst_cand[3] = acc[5].round_inplace();
        __syncwarp(tm);
    }
}

// Staging of a run and its halo block, or 0 when it would crowd the SM.
__host__ __device__ inline size_t profile_stage_bytes(size_t elem, uint32_t N, size_t smem_before)
{
    const size_t bytes = ((size_t)(kRun + 1) * N * elem + 15) / 16 * 16;
    return (bytes <= 48 * 1024 && smem_before + bytes <= 100 * 1024) ? bytes : 0;
}

// Three float32 candidates with k >= 1 (FMA form, see the candidate loop)
// in one walk over the thread's groups: one load per group, the three JEE
// counters in the lanes of one register.  Every lane of the warp calls it.
template <typename Stage>
__device__ __forceinline__ void profile_chunk3(const TBlock<4> &b, int s, int ge, const uint32_t *codes,
                                               Stage *cs, int t)
{
    using lt = typename LaneT<4>::t;
    constexpr int H = DT_<4>::H;
    float bs[3];
    uint32_t qp[3], qpp[3];
    int64_t sq[3], sA[3], sB[3];
    // u = q - ca qp + cb qpp (S3: ca = -1 on the previous q)
    const uint32_t ca = s == 0 ? 0u : (s == 1 ? 1u : (s == 2 ? 2u : 0xffffffffu)),
                   cb = s == 2 ? 1u : 0u;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const Quant<4> Q((int)codes[j], b.Eb);
        bs[j] = Q.scale;
        const Carry c = carry_in<4>(b, QuantM<4, 1>(Q), 4 * b.g0);
        qp[j] = (s == 1 || s == 3) ? c.qp1 : c.qp2;
        qpp[j] = c.qpp2;
        sq[j] = sA[j] = sB[j] = 0;
    }
    Tok3 tk;
    tk.init();
    uint32_t o[3] = {0u, 0u, 0u};  // width terms of the current BFPE group
#pragma unroll 1
    for (int g = b.g0; g < ge; ++g) {
        lt xv[4];
        load4<4, true>(b, 4 * g, xv);
        const int nv = b.L - 4 * g;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float xf = __uint_as_float(xv[i]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float T = __fmaf_rn(xf, bs[j], 12582912.0f);
                const uint32_t q = (uint32_t)(__float_as_int(T) - 0x4B400000);
                o[j] |= bits_term((int32_t)(q - ca * qp[j] + cb * qpp[j]));
                qpp[j] = qp[j];
                qp[j] = q;
                const float r = __fmaf_rn(xf, bs[j], -__fsub_rn(T, 12582912.0f));
                const int32_t Dp = __float2int_rn(__fmul_rn(r, 16777216.0f));
                const int32_t qs = i < nv ? (int32_t)q : 0;
                sq[j] += qs;
                sA[j] += (int64_t)qs * qs;
                sB[j] += (int64_t)qs * Dp;
            }
        }
        // |u| < 2^25 here, so no width reaches 31
        if (!b.gsh || (g & 1)) {
            tk.push(32 - __clz(o[0]), 32 - __clz(o[1]), 32 - __clz(o[2]));
            o[0] = o[1] = o[2] = 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        int nib, sume;
        team_tokens<TS>(tk.lane(j), b.g0 == 0, nib, sume);
        const int64_t rq = team_sum_i64(sq[j]), rA = team_sum_i64(sA[j]), rB = team_sum_i64(sB[j]);
        if (t == 0) {
            cs[j].sq = rq;
            cs[j].A = rA;
            cs[j].B = rB;
            cs[j].D = 0;
            cs[j].bits = (uint32_t)H + 4u * (uint32_t)nib + (4u << b.gsh) * (uint32_t)sume;
            cs[j].fast = 1;
        }
    }
}

// One run (kRun consecutive blocks, a level-1 node of the summation tree):
// the CTA's teams take one block each and write the run's partial sums.
// INL: the run sizes the sum stream itself for the stream decision (the
// batched kernel); single-array kernels read a.sel instead.
template <int DT, bool INL>
__device__ __forceinline__ void profile_run(const ProfArgs &a, uint64_t run, uint8_t *psm)
{
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int H = T::H;
    const int team = threadIdx.x / TS, t = tlane<TS>();
    const int nteams = blockDim.x / TS;  // = kRun
    const int nc = a.ncand;
    const int Qn = 2 + 4 * nc;
    CandStage<DT> *cs = reinterpret_cast<CandStage<DT> *>(psm) + (size_t)team * nc;
    double *bv = reinterpret_cast<double *>(psm + (size_t)nteams * nc * sizeof(CandStage<DT>));
    long long *accmem = reinterpret_cast<long long *>(bv + (size_t)nteams * Qn);
    __shared__ uint32_t s_fb[kRun];   // fallback requests: bit 0 block, bit 1+i candidate i
    __shared__ int s_ok[kRun];
    __shared__ uint64_t s_txx[kRun][4];  // f32: sum x^2 of the tiny samples (side grid)

    const int gp = a.gp;
    const uint64_t j = run * nteams + team;
    const raw *x = reinterpret_cast<const raw *>(a.x);
    // the run's blocks and the one before it in shared memory: the sweep
    // passes over every block once per candidate
    uint64_t base = 0;
    if (a.stage_off) {
        raw *xs = reinterpret_cast<raw *>(psm + a.stage_off);
        const uint64_t jb0 = run * (uint64_t)nteams;
        base = jb0 ? jb0 - 1 : 0;
        const uint64_t bend = min(jb0 + (uint64_t)nteams, a.nb);
        if (stage_blocks<DT>(xs, x, a.n, a.N, base, bend > base ? bend : base, a.status, 1ll << 31))
            x = xs;  // else (a wait ran out) read the blocks from global memory
        else
            base = 0;
        __syncthreads();
    }
    int s;
    if (!INL && a.sel) {
        s = j < a.nb ? a.sel[j] : 0;
    } else {
        TBlock<DT> pv;
        open_team_block<DT, TS>(pv, x, a.n, a.N, a.nb, j == 0 ? 0 : j - 1, gp, base, a.gsh);
        s = team_best_stream<DT, TS>(pv, INL && a.sum != 0);
    }
    TBlock<DT> b;
    open_team_block<DT, TS>(b, x, a.n, a.N, a.nb, j, gp, base, a.gsh);
    const bool live = b.active && !b.bad;
    if (b.active && b.bad && t == 0) set_status(a.status, -8);
    const int ge = live ? b.g1 : b.g0;  // my groups [g0, ge)

    // ---- block sums of x and x^2
    double blk_x[2] = {0.0, 0.0};
    bool tiny = false;
    bool side = false;  // f32: block sums and sum d^2 on the 256-bit side grids
    i128 sxx128 = 0;   // f32: sum X^2, X = x 2^(47-Eb)
    W256 wxx;          // f64: window 2^(2Eb - kWin)
    w256_zero(wxx);
    if constexpr (DT == 4) {
        int64_t sx = 0;
        uint64_t hh = 0, hl = 0, ll = 0;  // X = xh 2^24 + xl: sums of xh^2, xh xl, xl^2
        const int bmax = b.Eb + 126;      // biased exponent of the block maximum
#pragma unroll 1
        for (int g = b.g0; g < ge; ++g) {
            lt xv[4];
            load4<DT>(b, 4 * g, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t v = (uint32_t)xv[i];
                if (4 * g + i >= b.L || !(v & 0x7fffffffu)) continue;
                const int bexp = (int)((v >> 23) & 0xff);
                const int sh = bexp - bmax + 23;  // X = M << sh
                if (sh < 0 || bexp == 0) {
                    tiny = true;
                    continue;
                }
                const uint64_t X = (uint64_t)((v & 0x7fffffu) | 0x800000u) << sh;
                sx += (v >> 31) ? -(int64_t)X : (int64_t)X;
                const uint64_t xh = X >> 24, xl = X & 0xffffffu;
                hh += xh * xh;
                hl += xh * xl;
                ll += xl * xl;
            }
        }
        const i128 mine = ((i128)hh << 48) + ((i128)hl << 25) + (i128)ll;
        sxx128 = team_sum_i128(mine);
        sx = team_sum_i64(sx);
        tiny = team_sum<TS>((int)tiny) > 0;
        // Samples below 2^(Eb-24) quantise to 0 at every power-of-two code, so
        // they enter only sum x, sum x^2 and sum d^2 = sum x^2: exact 256-bit
        // side sums on finer grids (LSB 2^(Eb-237) and 2^(2Eb-239)).
        if (__any_sync(kFull, tiny)) {
            W256 tx, txx;
            w256_zero(tx);
            w256_zero(txx);
            bool deep = false;  // below even the side grids
            if (tiny) {
#pragma unroll 1
                for (int i = 4 * b.g0; i < min(4 * ge, b.L); ++i) {
                    const uint32_t v = reinterpret_cast<const uint32_t *>(b.p)[i];
                    const int bexp = (int)((v >> 23) & 0xff);
                    if (!(v & 0x7fffffffu) || (bexp != 0 && bexp - bmax + 23 >= 0)) continue;
                    const int ex = (bexp ? bexp : 1) - 150;
                    const uint32_t Mt = (v & 0x7fffffu) | (bexp ? 0x800000u : 0u);
                    const int px = ex - (b.Eb - 237), pxx = 2 * ex - (2 * b.Eb - 239);
                    if (px < 0 || pxx < 0 || b.Eb < -80) {  // subnormal blocks: fallback
                        deep = true;
                        continue;
                    }
                    w256_add(tx, (u128)Mt, px, (v >> 31) != 0);
                    w256_add(txx, (u128)((uint64_t)Mt * Mt), pxx, false);
                }
            }
            tx = team_sum_w256(tx);
            txx = team_sum_w256(txx);
            deep = team_sum<TS>((int)deep) > 0;
            if (tiny && !deep) {
                if (t == 0) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) s_txx[team][i] = txx.l[i];  // tiny part only
                }
                w256_add(tx, (u128)(sx < 0 ? -sx : sx), 190, sx < 0);
                w256_add(txx, (u128)sxx128, 145, false);
                blk_x[0] = round_w256(tx, b.Eb - 237);
                blk_x[1] = round_w256(txx, 2 * b.Eb - 239);
                side = true;
            }
            tiny = deep;  // only these still need the exact fallback
        }
        if (!side) {
            blk_x[0] = round_i128((i128)sx, b.Eb - 47);
            blk_x[1] = round_i128(sxx128, 2 * b.Eb - 94);
        }
    } else if constexpr (DT == 5) {
        W256 wx;
        w256_zero(wx);
#pragma unroll 1
        for (int g = b.g0; g < ge; ++g) {
            lt xv[4];
            load4<DT>(b, 4 * g, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (4 * g + i >= b.L) continue;
                const FDec<DT> d = fdec<DT>(xv[i]);
                if (!d.M) continue;
                const int pxx = 2 * d.ex - (2 * b.Eb - kWin), px = d.ex - (b.Eb - kWin);
                if (pxx < 0) {
                    tiny = true;
                    continue;
                }
                w256_add(wxx, (u128)d.M * d.M, pxx, false);
                w256_add(wx, (u128)d.M, px, d.neg);
            }
        }
        wxx = team_sum_w256(wxx);
        wx = team_sum_w256(wx);
        tiny = team_sum<TS>((int)tiny) > 0;
        blk_x[0] = round_w256(wx, b.Eb - kWin);
        blk_x[1] = round_w256(wxx, 2 * b.Eb - kWin);
    } else {
        int64_t sx = 0;
        i128 sxx = 0;
#pragma unroll 1
        for (int g = b.g0; g < ge; ++g) {
            lt xv[4];
            load4<DT>(b, 4 * g, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (4 * g + i < b.L) {
                    sx += xv[i];
                    sxx += (i128)((int64_t)xv[i] * xv[i]);
                }
            }
        }
        sx = team_sum_i64(sx);
        sxx = team_sum_i128(sxx);
        blk_x[0] = round_i128(sx, 0);
        blk_x[1] = round_i128(sxx, 0);
    }

    // ---- candidates
    uint32_t fbmask = tiny ? 1u : 0u;
    // Codes that quantise every sample to 0 (code 4095, or k >= Q + 1 for
    // floats, |X| < 2^Q, and k >= W for integers, |x| <= 2^(W-1)): sums of
    // y, xy and y^2 are 0, sum d^2 is the block's sum x^2, and the packet has
    // every exponent 0 (the first absolute, then zero diffs two to a joint
    // token).  They need no pass over the block when the block's own sums
    // are exact (no fallback); the codes increase, so they end the list.
    constexpr int kZeroK = T::F ? T::Q + 1 : T::W;
    int ct = nc;
    while (ct > 0 && (a.codes[ct - 1] == 4095 || (int)(a.codes[ct - 1] >> 7) >= kZeroK)) --ct;
    uint32_t zeromask = 0;  // candidates taken as all-zero
    const uint32_t zero_bits =
        (uint32_t)H + 4u * (uint32_t)(2 + ((b.G >> b.gsh) > 0 ? (b.G >> b.gsh) / 2 : 0));
#pragma unroll 1
    for (int ci = 0; ci < nc; ++ci) {
        if (ci >= ct && __all_sync(kFull, !(fbmask & 1u) || !b.active)) {
            // warp-uniform: every team of the warp skips this candidate
            zeromask |= 1u << ci;
            if (t == 0) {
                cs[ci].sq = 0;
                cs[ci].A = 0;
                cs[ci].B = 0;
                cs[ci].D = 0;
                cs[ci].bits = zero_bits;
                cs[ci].fast = 1;
            }
            continue;
        }
        if constexpr (DT == 4) {
            // three float32 candidates in one walk (FMA form, all k >= 1, no
            // fallback); warp-uniform, so the team collectives stay in step
            if (ci + 3 <= ct) {
                bool ok = !tiny && b.Eb >= -80;
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    const int cd = (int)a.codes[ci + jj];
                    ok &= Quant<DT>(cd, b.Eb).mode == 1 && b.Eb + (cd >> 7) <= 127 &&
                          (cd & 127) == 0;
                }
                if (__all_sync(kFull, ok || !b.active)) {
                    profile_chunk3(b, s, ge, &a.codes[ci], cs + ci, t);
                    ci += 2;
                    continue;
                }
            }
        }
        const int code = (int)a.codes[ci];
        const int k = code >> 7;
        const Quant<DT> Q(code, b.Eb);
        const int s_exp = b.Eb - T::Q + k;
        const bool pow2 = (code & 127) == 0;
        bool fast = true;
        if constexpr (DT == 4) fast = pow2 && !tiny && b.Eb >= -80 && b.Eb + k <= 127 && Q.mode != 0;
        if constexpr (DT == 5) fast = pow2 && !tiny && s_exp >= T::EMIN_U && b.Eb + k <= T::EMAXV;
        // integers: the decoder's y = clamp(RNE(q R[m] 2^(k-24))), which is
        // q 2^k for m = 0
        [[maybe_unused]] const int64_t Rm = (int64_t)recip_entry(code & 127);
        TokCount tc;
        tc.init();
        int64_t sq = 0, sA = 0, sB = 0, sD = 0;  // 64-bit partials (f32, i8, i16)
        i128 wq = 0, wA = 0, wB = 0, wD = 0;     // 128-bit partials (f64, i32)
        with_quant<DT>(Q, [&](const auto &qf) {
            Stream1 sm(s, carry_in<DT>(b, qf, 4 * b.g0));
            [[maybe_unused]] const int cD = -103 - b.Eb - k;  // f32: D' shift = bexp + cD
            constexpr int QM = std::remove_reference_t<decltype(qf)>::kMode;
            if constexpr (DT == 4 && QM == 1) {
                // FMA form (k >= 1): T = x b + 1.5 2^23 rounded gives q; then
                // r = x b - q is exact in one FMA (|r| <= 1/2 within 24 bits)
                // and D' = r 2^24 is an integer whenever q != 0.
                const float bsc = Q.scale;
                uint32_t o = 0;  // width terms of the current BFPE group
#pragma unroll 1
                for (int g = b.g0; g < ge; ++g) {
                    lt xv[4];
                    load4<DT, true>(b, 4 * g, xv);
                    const int nv = b.L - 4 * g;  // samples of the block from here
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float xf = __uint_as_float(xv[i]);
                        const float T = __fmaf_rn(xf, bsc, 12582912.0f);
                        const uint32_t q = (uint32_t)(__float_as_int(T) - 0x4B400000);
                        const int32_t u = (int32_t)(q - sm.a * sm.qp + sm.bb * sm.qpp);
                        o |= bits_term(u);
                        sm.qpp = sm.qp;
                        sm.qp = q;
                        const float r = __fmaf_rn(xf, bsc, -__fsub_rn(T, 12582912.0f));
                        const int32_t Dp = __float2int_rn(__fmul_rn(r, 16777216.0f));
                        const int32_t qs = i < nv ? (int32_t)q : 0;  // padding adds nothing
                        sq += qs;
                        sA += (int64_t)qs * qs;
                        sB += (int64_t)qs * Dp;
                    }
                    if (!b.gsh || (g & 1)) {
                        tc.push(exp_from_or(o), true);
                        o = 0;
                    }
                }
            } else {
            uint32_t o = 0;  // width terms of the current BFPE group
#pragma unroll 1
            for (int g = b.g0; g < ge; ++g) {
                lt xv[4];
                load4<DT, true>(b, 4 * g, xv);
                int32_t qq[4], uu[4];
                o |= group1q<DT>(qf, xv, sm, qq, uu);
                if (!b.gsh || (g & 1)) {
                    tc.push(exp_from_or(o), true);
                    o = 0;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (4 * g + i >= b.L) continue;
                    const int32_t qi = qq[i];
                    if constexpr (DT == 4) {
                        const uint32_t v = (uint32_t)xv[i];
                        const uint32_t qm = (uint32_t)abs(qi);
                        const uint32_t M = (v & 0x7fffffu) | 0x800000u;
                        const int32_t Dm = (int32_t)(shl_clamp(M, (int)((v >> 23) & 0xff) + cD) - (qm << 24));
                        sq += qi;
                        sA += (int64_t)qm * qm;
                        sB += (int64_t)(int32_t)qm * Dm;
                    } else if constexpr (DT == 5) {
                        if (qi) {
                            const FDec<DT> d = fdec<DT>(xv[i]);
                            const int sh = s_exp - d.ex;
                            const uint64_t qm = (uint64_t)(qi < 0 ? -(int64_t)qi : (int64_t)qi);
                            int64_t rem = 0;
                            if (sh > 0 && sh < 64) rem = (int64_t)(d.M - (qm << sh));
                            const int64_t Dp = (sh > 0 && sh <= 53) ? rem * ((int64_t)1 << (53 - sh)) : 0;
                            wq += qi;
                            wA += (i128)((int64_t)qi * qi);
                            wB += (i128)(int64_t)qm * Dp;
                        }
                    } else {
                        const int64_t xi = (int64_t)xv[i];
                        constexpr int64_t lo = DT == 1 ? -128 : (DT == 2 ? -32768 : -2147483648ll);
                        constexpr int64_t hi = DT == 1 ? 127 : (DT == 2 ? 32767 : 2147483647ll);
                        int64_t yv;
                        if (pow2) {
                            yv = (int64_t)qi * ((int64_t)1 << k);
                        } else if (qi == 0 || code == 4095) {
                            yv = 0;
                        } else {
                            // the decoder's arithmetic: |q| < 2^31 and R[m] < 2^25, so
                            // V fits 56 bits; k >= 24 scales up with saturation
                            const int64_t V = (int64_t)qi * Rm;
                            if (k <= 23) {
                                yv = rne_shift_s64(V, 24 - k);
                            } else {
                                const int sh2 = k - 24;
                                const int64_t lim = (int64_t)1 << (62 - sh2);
                                yv = V >= lim ? INT64_MAX
                                              : (V <= -lim ? INT64_MIN : V * ((int64_t)1 << sh2));
                            }
                        }
                        yv = yv < lo ? lo : (yv > hi ? hi : yv);
                        const int64_t dd = xi - yv;
                        if constexpr (DT == 3) {
                            wq += yv;
                            wA += (i128)(xi * yv);
                            wB += (i128)(yv * yv);
                            wD += (i128)dd * dd;
                        } else {
                            sq += yv;
                            sA += xi * yv;
                            sB += yv * yv;
                            sD += dd * dd;
                        }
                    }
                }
            }
            }
        });
        int nib, sume;
        team_tokens<TS>(tc, b.g0 == 0, nib, sume);
        const uint32_t bits = (uint32_t)H + 4u * (uint32_t)nib + (4u << b.gsh) * (uint32_t)sume;
        i128 rq, rA, rB, rD = 0;
        if constexpr (DT == 5 || DT == 3) {
            rq = team_sum_i128(wq);
            rA = team_sum_i128(wA);
            rB = team_sum_i128(wB);
            if constexpr (DT == 3) rD = team_sum_i128(wD);
        } else {
            rq = team_sum_i64(sq);
            rA = team_sum_i64(sA);
            rB = team_sum_i64(sB);
            if constexpr (!T::F) rD = team_sum_i64(sD);
        }
        if (t == 0) {
            cs[ci].sq = rq;
            cs[ci].A = rA;
            cs[ci].B = rB;
            cs[ci].D = rD;
            cs[ci].bits = bits;
            cs[ci].fast = fast;
        }
        if (T::F && !fast) fbmask |= 2u << ci;
    }
    __syncwarp();
    // ---- per candidate: round the block sums (thread t: candidates t, t+8, ...)
    double *mybv = bv + (size_t)team * Qn;
    if (t == 0) {
        mybv[0] = blk_x[0];
        mybv[1] = blk_x[1];
    }
    for (int ci = t; ci < nc; ci += TS) {
        const CandStage<DT> &st = cs[ci];
        const int k = (int)(a.codes[ci] >> 7);
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (live && ((zeromask >> ci) & 1u)) {
            v[3] = blk_x[1];  // d = x: the block's sum x^2, rounded once
        } else if (live) {
            if constexpr (DT == 4) {
                if (st.fast) {
                    const int s2 = b.Eb - 23 + k;
                    v[0] = round_i128(st.sq, s2);
                    v[2] = round_i128(st.A, 2 * s2);
                    v[1] = round_i128(st.A * ((i128)1 << 24) + st.B, 2 * s2 - 24);
                    // sum d^2 on the grid 2^(2Eb - 94): Sxx - A 2^(48+2k) - B 2^(25+2k)
                    const i128 dd = sxx128 - st.A * ((i128)1 << (48 + 2 * k)) -
                                    st.B * ((i128)1 << (25 + 2 * k));
                    if (side) {
                        // dd (>= 0) is the exact sum d^2 of the other samples
                        W256 w;
#pragma unroll
                        for (int i = 0; i < 4; ++i) w.l[i] = s_txx[team][i];
                        w256_add(w, (u128)dd, 145, false);
                        v[3] = round_w256(w, 2 * b.Eb - 239);
                    } else {
                        v[3] = round_i128(dd, 2 * b.Eb - 94);
                    }
                }
            } else if constexpr (DT == 5) {
                if (st.fast) {
                    const int s2 = b.Eb - T::Q + k;
                    v[0] = round_i128(st.sq, s2);
                    v[2] = round_i128(st.A, 2 * s2);
                    v[1] = round_i128(st.A * ((i128)1 << T::P) + st.B, 2 * s2 - T::P);
                    W256 dd = wxx;
                    const int base = 2 * b.Eb - kWin;
                    const int pA = 2 * s2 - base, pB = 2 * s2 - T::P + 1 - base;
                    w256_add(dd, (u128)st.A, pA, true);
                    const bool bneg = st.B < 0;
                    w256_add(dd, (u128)(bneg ? -st.B : st.B), pB, !bneg);
                    v[3] = round_w256(dd, base);
                }
            } else {
                v[0] = round_i128(st.sq, 0);
                v[1] = round_i128(st.A, 0);
                v[2] = round_i128(st.B, 0);
                v[3] = round_i128(st.D, 0);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) mybv[2 + 4 * ci + q] = v[q];
    }
    if (t == 0) {
        s_fb[team] = live ? fbmask : 0u;
        s_ok[team] = b.active;
    }
    __syncthreads();
    // ---- exact fallbacks, one team at a time (rare)
    if constexpr (T::F) {
        for (int tm = 0; tm < nteams; ++tm) {
            const uint32_t req = s_fb[tm];
            if (!req) continue;
            const bool me = team == tm;
            if (req & 1u) fallback_team<DT>(b, 0, true, false, accmem, mybv, nullptr, me);
            for (int ci = 0; ci < nc; ++ci) {
                if (!((req >> (ci + 1)) & 1u)) continue;
                fallback_team<DT>(b, (int)a.codes[ci], false, true, accmem, nullptr,
                                  mybv + 2 + 4 * ci, me);
            }
            __syncthreads();
        }
    }
    // ---- the run's partials: sums over the CTA's blocks in block order
    for (int q = threadIdx.x; q < Qn; q += blockDim.x) {
        double acc = 0.0;
        for (int tm = 0; tm < nteams; ++tm)
            if (s_ok[tm]) acc = __dadd_rn(acc, bv[(size_t)tm * Qn + q]);
        a.run_sums[run * Qn + q] = acc;
    }
    for (int ci = threadIdx.x; ci < nc; ci += blockDim.x) {
        unsigned long long by = 0;
        for (int tm = 0; tm < nteams; ++tm)
            if (s_ok[tm]) {
                const uint32_t bt = reinterpret_cast<CandStage<DT> *>(psm)[(size_t)tm * nc + ci].bits;
                by += 4ull * ((bt + 31u) >> 5);
            }
        atomicAdd(a.bytes + ci, by);
    }
}

template <int DT>
__global__ void __launch_bounds__(128) k_profile(ProfArgs a)
{
    extern __shared__ __align__(16) uint8_t psm[];
    profile_run<DT, false>(a, a.run0 + blockIdx.x, psm);
}

// The runs of [run0, run1) that the one-block-per-thread sweep marked (rare
// blocks it does not cover exactly): the team sweep, CTAs striding over the
// range.
template <int DT>
__global__ void __launch_bounds__(128) k_profile_fix(ProfArgs a)
{
    extern __shared__ __align__(16) uint8_t psm[];
    // This CTA's runs are r0 + i gridDim.x.  The flags of blockDim.x of them
    // are read together (most sweeps flag none), and only a chunk with a
    // flagged run is walked run by run.
    const uint64_t stride = gridDim.x;
    for (uint64_t r0 = a.run0 + blockIdx.x; r0 < a.run1; r0 += stride * blockDim.x) {
        const uint64_t r = r0 + stride * threadIdx.x;
        if (!__syncthreads_or(r < a.run1 && a.run_flags[r])) continue;
        for (uint64_t rr = r0; rr < a.run1 && rr < r0 + stride * blockDim.x; rr += stride) {
            if (a.run_flags[rr]) profile_run<DT, false>(a, rr, psm);
            __syncthreads();
        }
    }
}

__device__ double corr_r(double sxx, double sxy, double syy)
{
    // sums beyond binary64 give a quiet NaN with a fixed bit pattern
    if (!isfinite(sxx) || !isfinite(sxy) || !isfinite(syy))
        return __longlong_as_double(0x7ff8000000000000ll);
    if (sxx == 0.0 && syy == 0.0) return 1.0;
    if (sxx == 0.0 || syy == 0.0) return 0.0;
    const double p = __dmul_rn(sxx, syy);
    if (isfinite(p) && p >= 2.2250738585072014e-308) return __ddiv_rn(sxy, __dsqrt_rn(p));
    return __ddiv_rn(__ddiv_rn(sxy, __dsqrt_rn(sxx)), __dsqrt_rn(syy));
}

// Points and summary from the sums of the whole array (threads 0..31).
__device__ void finalize_points(const ProfArgs &a, const double *tot, uint64_t container_fixed,
                                double *s_r)
{
    const int nc = a.ncand;
    const int i = threadIdx.x;
    if (i < nc) {
        apax_profile_point p;
        p.code = a.codes[i];
        p.bytes = container_fixed + *(volatile unsigned long long *)(a.bytes + i);
        p.sx = tot[0];
        p.sxx = tot[1];
        p.sy = tot[2 + 4 * i];
        p.sxy = tot[2 + 4 * i + 1];
        p.syy = tot[2 + 4 * i + 2];
        p.sdd = tot[2 + 4 * i + 3];
        p.r = corr_r(p.sxx, p.sxy, p.syy);
        p.flags = p.r >= a.target ? 1u : 0u;
        a.points[i] = p;
        s_r[i] = p.r;
    }
    __syncthreads();
    if (i == 0) {
        int rec = -1;
        for (int c = 0; c < nc; ++c) {
            if (s_r[c] >= a.target) rec = c;
            else break;
        }
        apax_profile_summary sm;
        sm.status = *(volatile int *)a.status;
        sm.recommended = rec < 0 ? 0 : rec;
        sm.recommended_code = a.codes[rec < 0 ? 0 : rec];
        sm.flags = rec < 0 ? 1u : 0u;
        sm.n = a.n;
        *a.summary = sm;
    }
}

// The levels of the fan-in-16 tree above `in` (cnt values per quantity;
// the next level goes to scratch buffer pi) and the finalisation, by one
// CTA.  Level by level, each value the in-order sum of 16 (or fewer) below it.
__device__ void tree_rest_cta(const ProfArgs &a, const double *in, uint64_t cnt, int pi, double *s_r)
{
    const int Qn = 2 + 4 * a.ncand;
    double *bufs[2] = {a.scratch, a.scratch + ((a.nruns + 15) / 16 + 1) * (uint64_t)Qn};
    while (cnt > 1) {
        const uint64_t nodes = (cnt + 15) / 16;
        for (uint64_t m = threadIdx.x; m < nodes * (uint64_t)Qn; m += blockDim.x) {
            const uint64_t node = m / Qn, q = m % Qn;
            const uint64_t a0 = node * 16, a1 = min(a0 + 16, cnt);
            double sum = __ldcg(in + a0 * Qn + q);
            for (uint64_t i = a0 + 1; i < a1; ++i) sum = __dadd_rn(sum, __ldcg(in + i * Qn + q));
            __stcg(bufs[pi] + node * Qn + q, sum);
        }
        __syncthreads();
        in = bufs[pi];
        pi ^= 1;
        cnt = nodes;
    }
    __syncthreads();
    // the totals into shared memory (at most 2 + 4 * 32 values)
    __shared__ double s_tot[2 + 4 * 32];
    for (int q = threadIdx.x; q < Qn; q += blockDim.x) s_tot[q] = __ldcg(in + q);
    __syncthreads();
    const uint64_t fixed = 40 + ((4 * a.nb + 7) / 8) * 8;
    finalize_points(a, s_tot, fixed, s_r);
}

// The whole tree over the array's run sums and the finalisation, by one CTA
// (after every run of the array is written).
__device__ void tree_finalize_cta(const ProfArgs &a, double *s_r)
{
    const int Qn = 2 + 4 * a.ncand;
    const double *in = a.run_sums;
    if (a.nruns == 0) {
        for (int q = threadIdx.x; q < Qn; q += blockDim.x) __stcg(a.scratch + q, 0.0);
        __syncthreads();
        in = a.scratch;
    }
    tree_rest_cta(a, in, a.nruns, 0, s_r);
}

// Small arrays (at most 256 runs): the tree and the finalisation in one CTA.
__global__ void __launch_bounds__(256) k_tree_one(ProfArgs a)
{
    __shared__ double s_r[32];
    tree_finalize_cta(a, s_r);
}

// Larger arrays: the tree's first level by every CTA (grid-stride over
// nodes x quantities), the levels above it and the finalisation by the CTA
// that finishes last (a.done counts finished CTAs; cleared by the call).
// One launch where the level-by-level kernels took one per level plus one.
__global__ void __launch_bounds__(256) k_tree_fused(ProfArgs a)
{
    __shared__ double s_r[32];
    __shared__ bool s_last;
    const int Qn = 2 + 4 * a.ncand;
    const uint64_t cnt = a.nruns, nodes = (cnt + 15) / 16;
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < nodes * (uint64_t)Qn;
         m += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t node = m / Qn, q = m % Qn;
        const uint64_t a0 = node * 16, a1 = min(a0 + 16, cnt);
        double sum = __ldcg(a.run_sums + a0 * Qn + q);
        for (uint64_t i = a0 + 1; i < a1; ++i) sum = __dadd_rn(sum, __ldcg(a.run_sums + i * Qn + q));
        __stcg(a.scratch + node * Qn + q, sum);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        tree_rest_cta(a, a.scratch, nodes, 1, s_r);
    }
}

template <int DT>
__device__ __noinline__ void profile_run_call(const ProfArgs &a, uint64_t run, uint8_t *psm)
{
    profile_run<DT, true>(a, run, psm);
}

// Many arrays' profiler sweeps in one persistent launch: global run
// tickets, owning array by binary search; the CTA that completes an array's
// last run adds up its tree and writes its points and summary.
__global__ void __launch_bounds__(128) k_profile_batch(ProfBatchArgs ba)
{
    extern __shared__ __align__(16) uint8_t psm[];
    __shared__ uint64_t s_run;
    __shared__ int s_job, s_last;
    __shared__ __align__(16) ProfArgs s_args;
    __shared__ double s_r[32];
    while (true) {
        if (threadIdx.x == 0) {
            const uint64_t g = atomicAdd(ba.ticket, 1ull);
            int lo = 0, hi = ba.count;
            if (g < ba.total_runs) {
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (ba.run_prefix[mid] <= g) lo = mid;
                    else hi = mid;
                }
                s_run = g - ba.run_prefix[lo];
            } else {
                s_run = ~0ull;
            }
            s_job = lo;
        }
        __syncthreads();
        if (s_run == ~0ull) break;
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(ba.jobs + s_job);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(ProfArgs) / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (s_args.nruns) {
            switch (s_args.dtype) {
            case 1: profile_run_call<1>(s_args, s_run, psm); break;
            case 2: profile_run_call<2>(s_args, s_run, psm); break;
            case 3: profile_run_call<3>(s_args, s_run, psm); break;
            case 4: profile_run_call<4>(s_args, s_run, psm); break;
            default: profile_run_call<5>(s_args, s_run, psm); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const uint64_t units = s_args.nruns ? s_args.nruns : 1;
            s_last = atomicAdd(s_args.done, 1u) == units - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            tree_finalize_cta(s_args, s_r);
        }
        __syncthreads();
    }
}

template <int DT>
cudaError_t launch_prof_dt(const ProfArgs &a, cudaStream_t s)
{
    const int threads = TS * kRun;
    const int Qn = 2 + 4 * a.ncand;
    size_t smem = (size_t)kRun * a.ncand * sizeof(CandStage<DT>) + (size_t)kRun * Qn * 8 +
                  (DT_<DT>::F ? (size_t)6 * PS<DT>::ND * 8 : 0);
    ProfArgs b = a;
    // the run and its halo block in shared memory (17 passes over a block)
    const size_t sb = profile_stage_bytes(sizeof(typename DT_<DT>::raw), a.N, smem);
    b.stage_off = sb ? (uint32_t)((smem + 15) / 16 * 16) : 0;
    if (sb) smem = b.stage_off + sb;
    if constexpr (DT == 4) {
        if (profile_t1_eligible(a)) {
            cudaError_t e = launch_profile_t1(b, s);
            if (e != cudaSuccess) return e;
            e = smem_limit<k_profile_fix<DT>>(smem);
            if (e != cudaSuccess) return e;
            const uint64_t runs = a.run1 - a.run0, cap = 2ull * (uint64_t)sm_count();
            if (runs) k_profile_fix<DT><<<(unsigned)(runs < cap ? runs : cap), threads, smem, s>>>(b);
            return cudaGetLastError();
        }
    }
    auto k = k_profile<DT>;
    const cudaError_t e = smem_limit<k_profile<DT>>(smem);
    if (e != cudaSuccess) return e;
    if (a.run1 > a.run0) k<<<(unsigned)(a.run1 - a.run0), threads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

size_t profile_smem(int ncand, bool any_float, int dtype_max_nd)
{
    const int Qn = 2 + 4 * ncand;
    (void)any_float;
    return (size_t)kRun * ncand * sizeof(CandStage<5>) + (size_t)kRun * Qn * 8 +
           (size_t)6 * dtype_max_nd * 8;
}

cudaError_t launch_profile_batch(const ProfBatchArgs &b, int max_ncand, unsigned ctas,
                                 cudaStream_t s)
{
    const size_t smem = profile_smem(max_ncand, true, PS<5>::ND);
    cudaError_t e = cudaFuncSetAttribute(k_profile_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (ctas) k_profile_batch<<<ctas, TS * kRun, smem, s>>>(b);
    return cudaGetLastError();
}

int profile_batch_occupancy(int max_ncand)
{
    const size_t smem = profile_smem(max_ncand, true, PS<5>::ND);
    int nb = 0;
    if (cudaFuncSetAttribute(k_profile_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_profile_batch, TS * kRun, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_profile_runs(const ProfArgs &a, cudaStream_t s)
{
    if (a.run0 > a.run1 || a.run1 > a.nruns) return cudaErrorInvalidValue;
    switch (a.dtype) {
    case 1: return launch_prof_dt<1>(a, s);
    case 2: return launch_prof_dt<2>(a, s);
    case 3: return launch_prof_dt<3>(a, s);
    case 4: return launch_prof_dt<4>(a, s);
    default: return launch_prof_dt<5>(a, s);
    }
}

cudaError_t launch_profile(const ProfArgs &a, cudaStream_t s)
{
    ProfArgs b = a;
    b.run0 = 0;
    b.run1 = a.nruns;
    cudaError_t e;
    if (a.sel) {  // the sum stream: every block's stream decision first
        SelArgs sa;
        sa.x = a.x;
        sa.n = a.n;
        sa.N = a.N;
        sa.nb = a.nb;
        sa.j0 = 0;
        sa.count = a.nb;
        sa.dtype = a.dtype;
        sa.gsh = a.gsh;
        sa.gp = 0;
        sa.sel = const_cast<uint8_t *>(a.sel);
        e = launch_best_streams(sa, s);
        if (e != cudaSuccess) return e;
    }
    e = launch_profile_runs(b, s);
    if (e != cudaSuccess) return e;
    return launch_profile_tree(b, s);
}

cudaError_t launch_profile_tree(const ProfArgs &a, cudaStream_t s)
{
    // a.done: the call's cleared completion counter (apax_profile's workspace)
    if (a.nruns <= 256) {
        k_tree_one<<<1, 256, 0, s>>>(a);
    } else {
        const uint64_t work = (a.nruns + 15) / 16 * (uint64_t)(2 + 4 * a.ncand);
        const uint64_t most = 4ull * (uint64_t)sm_count();
        const uint64_t ctas = (work + 255) / 256 < most ? (work + 255) / 256 : most;
        k_tree_fused<<<(unsigned)ctas, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace apax
