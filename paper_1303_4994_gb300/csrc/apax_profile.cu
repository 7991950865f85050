// apax_profile.cu -- profiler sweep (Sec. 4): for every candidate code, the
// exact fixed-quality packet sizes and the reconstruction sums of the decoded
// y against x, in one pass that reads the input once.
//
// One warp owns a run of 16 consecutive blocks (a level-1 node of the
// fan-in-16 summation tree).  Per block: the stream decision (code 0, one
// block lag, Sec. 6), then per candidate the quantised stream's exponents and
// JEE token count (packet size) and the exact block sums.
//
// Candidates are power-of-two attenuations a = 2^-k (codes with m = 0).  For
// floats, the decoded value is then exactly y = q 2^s with s = Eb - Q + k,
// so with the quantiser remainder d = x - y = D' 2^(s-P):
//   sum y    = 2^s  sum q
//   sum y^2  = 2^2s A,               A = sum q^2
//   sum xy   = 2^2s A + 2^(2s-P) B,  B = sum q D'
//   sum d^2  = sum x^2 - 2^2s A - 2^(2s-P+1) B
// all exact in 64/128/256-bit integers (sum x^2 in a 256-bit window anchored
// at the block maximum).  Blocks with values too small for the window, and
// candidates whose y leaves the normal range, take an exact fallback with a
// shared-memory superaccumulator.  Each block sum is rounded once to binary64
// and added into the run's partial in block order.
#include "apax_block.cuh"
#include "apax_exact.cuh"
#include "apax_kernels.h"

namespace apax {

namespace {

constexpr int kRun = 16;
constexpr int kWin = 200;  // window LSB = 2^(2 Eb - kWin) for sum x^2

__device__ __forceinline__ void set_status(int *st, int code) { atomicMin(st, code); }

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
    int bexp = (int)((v >> T::MB) & (B)T::EMAX);
    d.M = (uint64_t)(v & (((B)1 << T::MB) - 1)) | (bexp ? ((uint64_t)1 << T::MB) : 0);
    d.ex = (bexp ? bexp : 1) - T::BIAS - T::MB;
    d.neg = (v >> (sizeof(B) * 8 - 1)) & 1;
    return d;
}

// per-candidate staging (shared memory)
struct CandStage {
    i128 sq, A, B;   // float fast path partials, or int sums (sy, sxy, syy)
    i128 sdd;        // int path
    uint32_t bits;
    int fast;
    double fb[4];    // fallback results (sy, sxy, syy, sdd)
};

template <int DT>
struct ProfSmem {
    static constexpr bool F = DT_<DT>::F;
    static constexpr int ND = DT == 5 ? 144 : 26;
    static constexpr int LO = DT == 5 ? -2304 : -320;
};

// Exact fallback for one (block, candidate) or for the block-level sums.
// acc[0..5]: x, y, x^2, xy, y^2, d^2.
template <int DT>
__device__ void fallback_sums(const BlockView<DT> &b, int code, bool want_block, bool want_cand,
                              long long *accmem, double *out_block, double *out_cand)
{
    using T = DT_<DT>;
    using P = ProfSmem<DT>;
    SmemAcc<P::ND, P::LO> acc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        acc[i].d = accmem + i * P::ND;
        acc[i].clear();
    }
    const Code c(code);
    for (int ch = 0; ch < b.nch; ++ch) {
        typename LaneT<DT>::t x[8];
        chunk_x<DT>(b, ch, x);
        const int i0 = ch * kChunk + 8 * (int)lane_id();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (i0 + t >= b.L) continue;
            FDec<DT> dx = fdec<DT>(x[t]);
            const u128 xx = (u128)dx.M * dx.M;
            if (want_block) {
                acc[0].add(dx.M, dx.ex, dx.neg);
                acc[2].add(xx, 2 * dx.ex, false);
            }
            if (want_cand) {
                int32_t q = quantise<DT>(x[t], c, b.Eb);
                typename T::bits yb = q ? round_to_format<DT>((int64_t)q * (1ll << 24),
                                                               b.Eb - T::Q + c.k - 24)
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
    __syncwarp();
    const int l = (int)lane_id();
    // lanes round different accumulators in parallel
    double r = 0.0;
    if (want_block && l == 0) r = acc[0].round_inplace();
    if (want_block && l == 2) r = acc[2].round_inplace();
    if (want_cand && l == 1) r = acc[1].round_inplace();
    if (want_cand && l == 3) r = acc[3].round_inplace();
    if (want_cand && l == 4) r = acc[4].round_inplace();
    if (want_cand && l == 5) r = acc[5].round_inplace();
    double v0 = __shfl_sync(kFull, r, 0), v1 = __shfl_sync(kFull, r, 1),
           v2 = __shfl_sync(kFull, r, 2), v3 = __shfl_sync(kFull, r, 3),
           v4 = __shfl_sync(kFull, r, 4), v5 = __shfl_sync(kFull, r, 5);
    if (want_block) { out_block[0] = v0; out_block[1] = v2; }
    if (want_cand) { out_cand[0] = v1; out_cand[1] = v3; out_cand[2] = v4; out_cand[3] = v5; }
    __syncwarp();
}

template <int DT>
__global__ void __launch_bounds__(256) k_profile(ProfArgs a)
{
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    using PS = ProfSmem<DT>;
    constexpr int W = T::W, H = T::H;
    extern __shared__ uint8_t psm[];
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    const int nc = a.ncand;
    const size_t per_warp = (size_t)nc * sizeof(CandStage) + (PS::F ? 6 * PS::ND * 8 : 0);
    uint8_t *wsm = psm + (size_t)wid * ((per_warp + 15) & ~(size_t)15);
    CandStage *cs = reinterpret_cast<CandStage *>(wsm);
    long long *accmem = reinterpret_cast<long long *>(wsm + (size_t)nc * sizeof(CandStage));

    const uint64_t r = (uint64_t)blockIdx.x * wpc + wid;
    if (r < a.nruns) {
        const raw *x = reinterpret_cast<const raw *>(a.x);
        const uint64_t j0 = r * kRun, j1 = min(j0 + kRun, a.nb);
        int best_prev = 0;
        if (j0 > 0) {
            BlockView<DT> pv;
            open_block<DT>(pv, x, a.n, a.N, j0 - 1);
            best_prev = best_stream<DT>(pv);
        }
        double run_c[4] = {0.0, 0.0, 0.0, 0.0};  // lane i: candidate i
        double run_x[2] = {0.0, 0.0};
        unsigned long long run_bytes = 0;
        for (uint64_t j = j0; j < j1; ++j) {
            BlockView<DT> b;
            open_block<DT>(b, x, a.n, a.N, j);
            if (b.bad) {
                if (l == 0) set_status(a.status, -8);
                continue;
            }
            const int bj = best_stream<DT>(b);
            const int s = j == 0 ? bj : best_prev;
            best_prev = bj;
            double blk_x[2];
            bool tiny = false;
            W256 wxx;
            w256_zero(wxx);
            if constexpr (T::F) {
                // exact sum x and sum x^2 in 256-bit windows
                W256 wx;
                w256_zero(wx);
                for (int ch = 0; ch < b.nch; ++ch) {
                    lt xv[8];
                    chunk_x<DT>(b, ch, xv);
                    const int i0 = ch * kChunk + 8 * l;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if (i0 + t >= b.L) continue;
                        FDec<DT> d = fdec<DT>(xv[t]);
                        if (!d.M) continue;
                        const int pxx = 2 * d.ex - (2 * b.Eb - kWin), px = d.ex - (b.Eb - kWin);
                        if (pxx < 0) { tiny = true; continue; }
                        w256_add(wxx, (u128)d.M * d.M, pxx, false);
                        w256_add(wx, (u128)d.M, px, d.neg);
                    }
                }
                tiny = __any_sync(kFull, tiny);
                if (tiny) {
                    double dummy[4];
                    fallback_sums<DT>(b, 0, true, false, accmem, blk_x, dummy);
                } else {
                    wxx = warp_sum_w256(wxx);
                    W256 sx = warp_sum_w256(wx);
                    blk_x[0] = round_w256(sx, b.Eb - kWin);
                    blk_x[1] = round_w256(wxx, 2 * b.Eb - kWin);
                }
            } else {
                int64_t sx = 0;
                i128 sxx = 0;
                for (int ch = 0; ch < b.nch; ++ch) {
                    lt xv[8];
                    chunk_x<DT>(b, ch, xv);
                    const int i0 = ch * kChunk + 8 * l;
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (i0 + t < b.L) {
                            sx += xv[t];
                            sxx += (i128)((int64_t)xv[t] * xv[t]);
                        }
                }
                sx = warp_sum_i64(sx);
                sxx = warp_sum_i128(sxx);
                blk_x[0] = round_i128(sx, 0);
                blk_x[1] = round_i128(sxx, 0);
            }
            // candidates
            for (int ci = 0; ci < nc; ++ci) {
                const int code = (int)a.codes[ci];
                const int k = code >> 7;
                const Code c(code);
                int32_t p1 = 0, p2 = 0;
                int eprev = 0, nib = 0, sume = 0;
                bool carry = false;
                i128 acc_q = 0, acc_A = 0, acc_B = 0, acc_D = 0;
                const int s_exp = b.Eb - T::Q + k;
                bool fast = true;
                if constexpr (T::F) fast = !tiny && s_exp >= T::EMIN_U && b.Eb + k <= T::EMAXV;
                for (int ch = 0; ch < b.nch; ++ch) {
                    lt xv[8];
                    chunk_x<DT>(b, ch, xv);
                    const int i0 = ch * kChunk + 8 * l;
                    int32_t q[8];
                    int64_t sA = 0, sB = 0, sQ = 0;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const bool valid = i0 + t < b.L;
                        if constexpr (T::F) {
                            FDec<DT> d = fdec<DT>(xv[t]);
                            const int sh = s_exp - d.ex;
                            uint64_t qm = rne_shift_u64(d.M, sh);
                            int64_t rem = (sh > 0 && sh < 64) ? (int64_t)(d.M - (qm << sh)) : (sh >= 64 ? (int64_t)d.M : 0);
                            int32_t qs = d.neg ? -(int32_t)qm : (int32_t)qm;
                            q[t] = qs;
                            if (valid && qm) {
                                int64_t Dp = rem * ((int64_t)1 << (T::P - sh > 0 ? T::P - sh : 0));
                                if (d.neg) Dp = -Dp;
                                if constexpr (DT == 4) {
                                    sQ += qs;
                                    sA += (int64_t)qs * qs;
                                    sB += (int64_t)qs * Dp;
                                } else {
                                    acc_q += qs;
                                    acc_A += (i128)((int64_t)qs * qs);
                                    acc_B += (i128)qs * Dp;
                                }
                            }
                        } else {
                            int32_t qq = quantise<DT>(xv[t], c, 0);
                            q[t] = qq;
                            if (valid) {
                                int64_t yv = (int64_t)qq * ((int64_t)1 << k);
                                constexpr int64_t lo = DT == 1 ? -128 : (DT == 2 ? -32768 : -2147483648ll);
                                constexpr int64_t hi = DT == 1 ? 127 : (DT == 2 ? 32767 : 2147483647ll);
                                yv = yv < lo ? lo : (yv > hi ? hi : yv);
                                const int64_t xi = (int64_t)xv[t], dd = xi - yv;
                                if constexpr (DT == 3) {
                                    acc_q += yv;
                                    acc_A += (i128)(xi * yv);
                                    acc_B += (i128)(yv * yv);
                                    acc_D += (i128)((uint64_t)(dd < 0 ? -dd : dd) * (uint64_t)(dd < 0 ? -dd : dd));
                                } else {
                                    sQ += yv;
                                    sA += xi * yv;
                                    sB += yv * yv;
                                    acc_D += dd * dd;
                                }
                            }
                        }
                    }
                    if constexpr (DT != 5 && DT != 3) {
                        acc_q += sQ;
                        acc_A += sA;
                        acc_B += sB;
                    }
                    // padding past L, stream, exponents, tokens
                    const int last = b.L - 1;
                    if (last < (ch + 1) * kChunk) {
                        const int li = last - ch * kChunk;
                        const int32_t ql = __shfl_sync(kFull, q[li & 7], li >> 3);
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            if (i0 + t > last) q[t] = ql;
                    }
                    int gc = b.G - ch * 64;
                    gc = gc > 64 ? 64 : gc;
                    int32_t u1 = __shfl_up_sync(kFull, q[7], 1), u2 = __shfl_up_sync(kFull, q[6], 1);
                    if (l == 0) { u1 = p1; u2 = p2; }
                    int32_t u[8];
                    derive<W>(q, s, u1, u2, ch == 0 && l == 0, u);
                    const int g0 = 2 * l;
                    const int e0 = g0 < gc ? group_exp(u[0], u[1], u[2], u[3]) : 0;
                    const int e1 = g0 + 1 < gc ? group_exp(u[4], u[5], u[6], u[7]) : 0;
                    ChunkTok tk = chunk_tokens(e0, e1, gc, ch == 0, eprev, carry);
                    nib += tk.nib;
                    sume += __reduce_add_sync(kFull, (unsigned)(e0 + e1));
                    eprev = tk.last_e;
                    carry = tk.carry;
                    p1 = __shfl_sync(kFull, q[7], 31);
                    p2 = __shfl_sync(kFull, q[6], 31);
                }
                const uint32_t bits = (uint32_t)H + 4u * (uint32_t)nib + 4u * (uint32_t)sume;
                i128 rq = warp_sum_i128(acc_q), rA = warp_sum_i128(acc_A), rB = warp_sum_i128(acc_B);
                i128 rD = 0;
                if constexpr (!T::F) rD = warp_sum_i128(acc_D);
                if (l == 0) {
                    cs[ci].sq = rq;
                    cs[ci].A = rA;
                    cs[ci].B = rB;
                    cs[ci].sdd = rD;
                    cs[ci].bits = bits;
                    cs[ci].fast = fast;
                }
                if constexpr (T::F) {
                    if (!fast) {
                        double dummy[2];
                        fallback_sums<DT>(b, code, false, true, accmem, dummy, cs[ci].fb);
                    }
                }
            }
            __syncwarp();
            // lane ci finishes candidate ci: round the block sums to binary64
            if (l < nc) {
                const CandStage &st = cs[l];
                const int k = (int)(a.codes[l] >> 7);
                double v[4];
                if constexpr (T::F) {
                    if (st.fast) {
                        const int s2 = b.Eb - T::Q + k;
                        v[0] = round_i128(st.sq, s2);
                        v[2] = round_i128(st.A, 2 * s2);
                        v[1] = round_i128((st.A << T::P) + st.B, 2 * s2 - T::P);
                        W256 dd = wxx;
                        const int base = 2 * b.Eb - kWin;
                        const int pA = 2 * s2 - base, pB = 2 * s2 - T::P + 1 - base;
                        w256_add(dd, (u128)st.A, pA, true);
                        const bool bneg = st.B < 0;
                        w256_add(dd, (u128)(bneg ? -st.B : st.B), pB, !bneg);
                        v[3] = round_w256(dd, base);
                    } else {
                        v[0] = st.fb[0]; v[1] = st.fb[1]; v[2] = st.fb[2]; v[3] = st.fb[3];
                    }
                } else {
                    v[0] = round_i128(st.sq, 0);
                    v[1] = round_i128(st.A, 0);
                    v[2] = round_i128(st.B, 0);
                    v[3] = round_i128(st.sdd, 0);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) run_c[t] += v[t];
                run_bytes += pad32_bytes(st.bits);
            }
            run_x[0] += blk_x[0];
            run_x[1] += blk_x[1];
            __syncwarp();
        }
        const int Qn = 2 + 4 * nc;
        double *o = a.run_sums + r * (uint64_t)Qn;
        if (l == 0) { o[0] = run_x[0]; o[1] = run_x[1]; }
        if (l < nc) {
#pragma unroll
            for (int t = 0; t < 4; ++t) o[2 + 4 * l + t] = run_c[t];
            atomicAdd(a.bytes + l, run_bytes);
        }
    }
}

// One level of the fan-in-16 tree: out[m][q] = in[16m][q] + ... (in order).
__global__ void k_tree(const double *in, double *out, uint64_t cnt, int Qn)
{
    const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nodes = (cnt + 15) / 16;
    if (m >= nodes * (uint64_t)Qn) return;
    const uint64_t node = m / Qn, q = m % Qn;
    const uint64_t a0 = node * 16, a1 = min(a0 + 16, cnt);
    double s = in[a0 * Qn + q];
    for (uint64_t i = a0 + 1; i < a1; ++i) s = __dadd_rn(s, in[i * Qn + q]);
    out[node * Qn + q] = s;
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

__global__ void k_finalize(ProfArgs a, const double *tot, uint64_t container_fixed)
{
    const int nc = a.ncand;
    __shared__ int s_rec;
    if (threadIdx.x == 0) {
        int rec = -1;
        bool prefix = true;
        const int st = *a.status;
        for (int i = 0; i < nc; ++i) {
            apax_profile_point p;
            p.code = a.codes[i];
            p.bytes = container_fixed + a.bytes[i];
            p.sx = tot[0];
            p.sxx = tot[1];
            p.sy = tot[2 + 4 * i];
            p.sxy = tot[2 + 4 * i + 1];
            p.syy = tot[2 + 4 * i + 2];
            p.sdd = tot[2 + 4 * i + 3];
            p.r = corr_r(p.sxx, p.sxy, p.syy);
            p.flags = p.r >= a.target ? 1u : 0u;
            if (prefix && p.r >= a.target) rec = i;
            else prefix = false;
            a.points[i] = p;
        }
        apax_profile_summary sm;
        sm.status = st;
        sm.recommended = rec < 0 ? 0 : rec;
        sm.recommended_code = a.codes[rec < 0 ? 0 : rec];
        sm.flags = rec < 0 ? 1u : 0u;
        sm.n = a.n;
        *a.summary = sm;
        s_rec = rec;
    }
}

template <int DT>
cudaError_t launch_prof_dt(const ProfArgs &a, cudaStream_t s)
{
    using PS = ProfSmem<DT>;
    const int wpc = 8;
    const size_t per_warp = (size_t)a.ncand * sizeof(CandStage) + (PS::F ? 6 * PS::ND * 8 : 0);
    const size_t smem = (size_t)wpc * ((per_warp + 15) & ~(size_t)15);
    auto k = k_profile<DT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((a.nruns + wpc - 1) / wpc);
    if (grid) k<<<grid, 32 * wpc, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_profile(const ProfArgs &a, cudaStream_t s)
{
    cudaError_t e;
    switch (a.dtype) {
    case 1: e = launch_prof_dt<1>(a, s); break;
    case 2: e = launch_prof_dt<2>(a, s); break;
    case 3: e = launch_prof_dt<3>(a, s); break;
    case 4: e = launch_prof_dt<4>(a, s); break;
    default: e = launch_prof_dt<5>(a, s); break;
    }
    if (e != cudaSuccess) return e;
    // upper levels of the fan-in-16 tree
    const int Qn = 2 + 4 * a.ncand;
    uint64_t cnt = a.nruns;
    const double *in = a.run_sums;
    double *bufs[2] = {a.scratch, a.scratch + ((a.nruns + 15) / 16 + 1) * (uint64_t)Qn};
    int pi = 0;
    if (cnt == 0) {
        e = cudaMemsetAsync(a.scratch, 0, sizeof(double) * Qn, s);
        if (e != cudaSuccess) return e;
        in = a.scratch;
    }
    while (cnt > 1) {
        const uint64_t nodes = (cnt + 15) / 16;
        const uint64_t threads = nodes * Qn;
        k_tree<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(in, bufs[pi], cnt, Qn);
        in = bufs[pi];
        pi ^= 1;
        cnt = nodes;
    }
    const uint64_t nb = a.nb;
    const uint64_t fixed = 40 + ((4 * nb + 7) / 8) * 8;
    k_finalize<<<1, 32, 0, s>>>(a, in, fixed);
    return cudaGetLastError();
}

}  // namespace apax
