// apax_encode_res.cu -- the fixed-quality block encoder (Sec. 6) with each
// team's block held in registers, for blocks of at most 256 samples of
// int8, int16 and float32 (teams of 8 threads, at most 8 groups of 4
// samples a thread).
//
// The general tile (apax_encode.cu) reads a block five times: its
// predecessor twice (the block maximum and the code-0 stream sizes of the
// one-block-lag decision) and itself three times (maximum, exponents,
// mantissas), the repeats from L2.  Here every team loads its own block once,
// with the padding of Sec. 6 packets already in place, and every pass runs on
// the registers:
//   1. the block maximum (float block exponent);
//   2. its own code-0 stream sizes, i.e. the decision its successor uses;
//      warp 0 also sizes the block before the tile (the halo), as one team
//      of 32 so that the other warps' wait at the barrier is short;
//   3. after one CTA barrier, the stream of block j is the decision of team
//      j - 1 (block 0 keeps its own);
//   4. exponents and JEE tokens at the given code, then the mantissas, into
//      the team's packet image in shared memory, and out with coalesced
//      stores -- as in the general tile, with the same decoupled look-back
//      over tiles for the packet offsets.
// Carries across a team's threads (the previous samples that the derivative
// streams need) come by shuffle from the neighbouring thread's registers.
// Containers with the sum stream take their decisions from the pre-pass
// (a.sel).  The bytes are the general tile's.
#include "apax_team.cuh"
#include "apax_kernels.h"
#include "apax_encode.cuh"

namespace apax {

namespace {

constexpr int kTS = 8;  // threads per block
constexpr int kGM = 8;  // groups of 4 per thread at most (N <= 256)

template <int DT>
using Regs = typename LaneT<DT>::t[kGM][4];

// The carries entering my first group at the current code: from the
// previous thread's last two samples, or the block start (see carry_in).
// q2, q3: my last group's samples 2 and 3 quantised; qs: the block's first
// sample quantised (meaningful on thread 0).  Warp-collective.
__device__ __forceinline__ Carry res_carry(uint32_t q2, uint32_t q3, uint32_t qs, int t)
{
    const uint32_t p2 = tshfl_up<kTS>(q2, 1), p3 = tshfl_up<kTS>(q3, 1);
    Carry c;
    if (t == 0) {
        c.qp1 = 0;
        c.qp2 = qs;
        c.qpp2 = 2u * qs;
    } else {
        c.qp1 = p3;
        c.qp2 = p3;
        c.qpp2 = p2;
    }
    return c;
}

// The quantised samples that res_carry needs, at quantiser Q: v2, v3 are my
// last group's samples 2 and 3 (kept at load time: picking them out of xr by
// a run-time index would move xr to local memory).
template <int DT>
__device__ __forceinline__ Carry res_carry_at(const Quant<DT> &Q, const Regs<DT> &xr,
                                              typename LaneT<DT>::t v2, typename LaneT<DT>::t v3, int t)
{
    uint32_t q2 = 0, q3 = 0, qs = 0;
    with_quant<DT>(Q, [&](const auto &qf) {
        q2 = (uint32_t)qf(v2);
        q3 = (uint32_t)qf(v3);
        qs = (uint32_t)qf(xr[0][0]);
    });
    return res_carry(q2, q3, qs, t);
}

// Stream s at code Q over my groups: the greedy token counter and each BFPE
// group's exponent in ebuf[g >> gsh].  The stream values replace the samples
// in xr (the mantissa writer reads them there).
template <int DT>
__device__ __forceinline__ TokCount res_pass(const TBlock<DT> &b, Regs<DT> &xr, const Quant<DT> &Q,
                                             const Carry &c, int s, uint8_t *ebuf)
{
    TokCount tc;
    tc.init();
    const int ng = b.g1 - b.g0;
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 st(s, c);
        uint32_t acc = 0;
#pragma unroll
        for (int i = 0; i < kGM; ++i) {
            if (i < ng) {
                int32_t u[4];
                acc |= group1<DT>(qf, xr[i], st, u);
#pragma unroll
                for (int k = 0; k < 4; ++k) xr[i][k] = (typename LaneT<DT>::t)u[k];
                const int g = b.g0 + i;
                if (!b.gsh || (g & 1)) {
                    const int e = exp_from_or(acc);
                    ebuf[g >> b.gsh] = (uint8_t)e;
                    tc.push(e, true);
                    acc = 0;
                }
            }
        }
    });
    return tc;
}

// The best of S0-S2 at code 0 on the registers.  Warp-collective.
template <int DT>
__device__ __forceinline__ int res_best_stream(const TBlock<DT> &b, const Regs<DT> &xr,
                                               typename LaneT<DT>::t l2, typename LaneT<DT>::t l3, int t)
{
    const Quant<DT> Q(0, b.Eb);
    Carry c = res_carry_at<DT>(Q, xr, l2, l3, t);
    Tok3 tk;
    tk.init();
    const int ng = b.g1 - b.g0;
    with_quant<DT>(Q, [&](const auto &qf) {
        uint32_t a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int i = 0; i < kGM; ++i) {
            if (i < ng) {
                uint32_t o0, o1, o2;
                group3<DT>(qf, xr[i], c, o0, o1, o2);
                a0 |= o0;
                a1 |= o1;
                a2 |= o2;
                if (!b.gsh || ((b.g0 + i) & 1)) {
                    tk.push(exp_from_or(a0), exp_from_or(a1), exp_from_or(a2));
                    a0 = a1 = a2 = 0;
                }
            }
        }
    });
    uint32_t bits[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int nib, sume;
        team_tokens<kTS>(tk.lane(k), b.g0 == 0, nib, sume);
        bits[k] = 4u * (uint32_t)nib + (4u << b.gsh) * (uint32_t)sume;
    }
    int s = 0;
    if (bits[1] < bits[s]) s = 1;
    if (bits[2] < bits[s]) s = 2;
    return s;
}

template <int DT>
__device__ __forceinline__ void encode_tile_res(const EncArgs &a, uint64_t tile, uint32_t *smem)
{
    __shared__ uint32_t s_words[32];
    __shared__ uint32_t s_total;
    __shared__ uint64_t s_base;
    __shared__ int s_dec[32];
    __shared__ int s_halo;
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int H = T::H, TS = kTS;
    const int team = threadIdx.x / TS, t = tlane<TS>();
    const int nteams = blockDim.x / TS;
    const int gp = a.gp;  // <= kGM

    const uint64_t jb = a.jb0 + tile * (uint64_t)nteams;  // the tile's first block
    const uint64_t j = jb + (uint64_t)team;
    const uint64_t jl = j - a.jb0, nbl = a.nb - a.jb0;
    int code = (int)a.code;
    if (a.code_dev) code = (int)*a.code_dev;
    uint32_t *pkt = smem + (size_t)team * (a.pkt_words + a.ebuf_words);
    uint8_t *ebuf = reinterpret_cast<uint8_t *>(pkt + a.pkt_words);
    if (tile == 0 && threadIdx.x == 0) write_container_header(a, code);
    const raw *x = reinterpret_cast<const raw *>(a.x);

    // ---- 1. my groups of the block into registers (load4's padding)
    TBlock<DT> b;
    b.active = j < a.nb;
    const uint64_t off = j * (uint64_t)a.N;
    b.p = x + (b.active ? off : 0);
    b.L = b.active ? (int)((a.n - off) < a.N ? (a.n - off) : a.N) : 0;
    b.gsh = a.gsh;
    b.G = b.gsh ? 2 * ((b.L + 7) >> 3) : (b.L + 3) >> 2;
    b.g0 = t * gp;
    b.g1 = min(b.g0 + gp, b.G);
    b.Eb = 0;
    b.bad = false;
    lt xr[kGM][4];
    lt l2 = 0, l3 = 0;  // my last group's samples 2 and 3
#pragma unroll
    for (int i = 0; i < kGM; ++i) {
        if (i < gp && b.g0 + i < b.G) {
            load4<DT, true>(b, 4 * (b.g0 + i), xr[i]);
            l2 = xr[i][2];
            l3 = xr[i][3];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) xr[i][k] = 0;
        }
    }
    if constexpr (T::F) {
        // the largest magnitude's bit pattern (NaN and infinities compare
        // above every finite magnitude); padding repeats a sample
        using B = typename T::bits;
        constexpr B absm = ~((B)1 << (sizeof(B) * 8 - 1));
        constexpr B expm = (B)T::EMAX << T::MB;
        B mx = 0;
#pragma unroll
        for (int i = 0; i < kGM; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const B v = (B)xr[i][k] & absm;
                mx = v > mx ? v : mx;
            }
#pragma unroll
        for (int m = TS / 2; m >= 1; m >>= 1) {
            const B o = tshfl_xor<TS>(mx, m);
            mx = o > mx ? o : mx;
        }
        b.bad = mx >= expm;
        b.Eb = b.bad ? 0 : block_exp_from_maxbits<DT>((uint64_t)mx);
    }
    if (b.active && b.bad && t == 0) set_status(a.status, -8);

    // ---- 2-3. stream decisions: my block's own (its successor's stream),
    // the halo before the tile, then block j takes block j - 1's
    int s;
    if (a.sel) {
        s = jl < nbl ? a.sel[jl] : 0;
    } else {
        const int own = res_best_stream<DT>(b, xr, l2, l3, t);
        if (t == 0) s_dec[team] = own;
        if (threadIdx.x < 32) {
            // warp 0, as one team of 32: the block before the tile (the
            // other warps wait for it at the barrier, so all its lanes share it)
            TBlock<DT> pv;
            const bool halo = jb > 0 && jb < a.nb;
            const int gp32 = b.gsh ? 2 * (int)((a.N / 8 + 31) / 32) : (int)((a.N / 4 + 31) / 32);
            open_team_block<DT, 32>(pv, x, a.n, a.N, halo ? a.nb : 0, halo ? jb - 1 : 0, gp32, 0,
                                    a.gsh);
            const int hs = team_best_stream<DT, 32>(pv, false);
            if (threadIdx.x == 0) s_halo = hs;
        }
        __syncthreads();
        s = j == 0 ? own : (team == 0 ? s_halo : s_dec[team - 1]);
    }

    // ---- 4. exponents and tokens at the code, then the packet
    const Quant<DT> Q(code, b.Eb);
    const Carry cq = res_carry_at<DT>(Q, xr, l2, l3, t);
    const TokCount tc = res_pass<DT>(b, xr, Q, cq, s, ebuf);  // xr now holds the stream values
    int nib_total, sume_total, nib_mine;
    bool s_in;
    team_tokens<TS>(tc, b.g0 == 0, nib_total, sume_total, &s_in, &nib_mine);
    const uint32_t wm = 4u << b.gsh;  // mantissa bits per exponent unit
    const uint32_t bits = (uint32_t)H + 4u * (uint32_t)nib_total + wm * (uint32_t)sume_total;
    const uint32_t plen = pad32_bytes(bits);
    const uint32_t words = b.active ? plen >> 2 : 0;
    {
        // the tile's size: scan it and publish the aggregate now
        if (t == 0) s_words[team] = words;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const uint32_t v = l < nteams ? s_words[l] : 0;
            const uint32_t incl = warp_incl_scan(v);
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            __syncwarp();
            if (l < nteams) s_words[l] = incl - v;
            if (l == 0) {
                s_total = total;
                publish_aggregate(a, tile, total);
            }
        }
    }
    for (uint32_t w = t; w < words; w += TS) pkt[w] = 0;
    __syncwarp();
    const int nib_before = team_incl_scan<TS>(nib_mine) - nib_mine;
    const int sume_before = team_incl_scan<TS>(tc.sume) - tc.sume;
    if (b.active) {
        if (t == 0) {
            atomicOr(&pkt[0], (uint32_t)s | ((uint32_t)code << 2) | (plen << 14));
            if (H == 48) atomicOr(&pkt[1], (uint32_t)(uint16_t)(int16_t)b.Eb);
        }
        NibWriter nw;
        nw.start(pkt, (uint32_t)H + 4u * (uint32_t)nib_before);
        write_tokens(nw, ebuf, 1, b.g0 >> b.gsh, b.g1 >> b.gsh, b.G >> b.gsh, s_in);
        nw.flush();
        NibWriter mw;
        mw.start(pkt, (uint32_t)H + 4u * (uint32_t)nib_total + wm * (uint32_t)sume_before);
        const int ng = b.g1 - b.g0;
#pragma unroll
        for (int i = 0; i < kGM; ++i) {
            if (i < ng) {
                const int32_t u[4] = {(int32_t)xr[i][0], (int32_t)xr[i][1], (int32_t)xr[i][2],
                                      (int32_t)xr[i][3]};
                write_group_fields(mw, ebuf[(b.g0 + i) >> b.gsh], u);
            }
        }
        mw.flush();
    }
    __syncthreads();

    // the packet's start in payload words: the look-back's exclusive prefix
    if (threadIdx.x < 32) {
        const uint64_t excl = lookback_prefix(a, tile, s_total);
        if (threadIdx.x == 0) s_base = excl;
    }
    __syncthreads();
    const uint64_t off_words = s_base + s_words[team];
    if (b.active) {
        const uint64_t start = a.poff + 4ull * off_words;
        if (t == 0) {
            if (off_words > 0xffffffffull) {
                set_status(a.status, -6);
            } else {
                reinterpret_cast<uint32_t *>(a.out + 40)[jl] = (uint32_t)off_words;
                if (jl == nbl - 1 && (nbl & 1)) reinterpret_cast<uint32_t *>(a.out + 40)[jl + 1] = 0;
            }
        }
        if (start + 4ull * words > a.cap) {
            if (t == 0) set_status(a.status, -5);
        } else {
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.out + start);
            for (uint32_t w = t; w < words; w += TS) dst[w] = pkt[w];
        }
    }

    // completion: the CTA that finishes the array's last tile writes the
    // payload size and the result
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done, 1u);
        if (prev == a.ntiles - 1) {
            __threadfence();
            volatile unsigned long long *last = a.tiles + (a.ntiles - 1);
            const uint64_t payload = 4ull * ((uint64_t)(*last) & kValMask);
            put_le(a.out + 28, payload, 8);
            volatile int *st = a.status;
            if (a.res) {
                a.res->bytes = a.poff + payload;
                a.res->status = *st;
            }
        }
    }
}

// Tiles in ticket order (the look-back needs every predecessor started).
template <int DT>
__global__ void __launch_bounds__(128) k_encode_res(EncArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint64_t s_tile;
    if (threadIdx.x == 0) s_tile = (uint64_t)atomicAdd(a.ticket, 1u);
    __syncthreads();
    encode_tile_res<DT>(a, s_tile, smem);
}

template <int DT>
cudaError_t launch_dt(const EncArgs &a, int threads, size_t smem, cudaStream_t s)
{
    const cudaError_t e = smem_limit<k_encode_res<DT>>(smem);
    if (e != cudaSuccess) return e;
    k_encode_res<DT><<<(unsigned)a.ntiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Fixed quality of int8, int16 and float32 blocks of at most 256 samples.
// (Fixed rate keeps the staged general tile: with the block in registers its
// search loops needed 168 registers a thread for float32; int32's exact
// quantiser needed 122, the general tile 56.)
bool encode_res_eligible(int dtype, int mode, uint32_t N, int ts)
{
    return ts == kTS && mode == APAX_FIXED_QUALITY && (dtype == 1 || dtype == 2 || dtype == 4) &&
           N <= (uint32_t)(4 * kTS * kGM);
}

cudaError_t launch_encode_res(const EncArgs &a, int threads, size_t smem, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, threads, smem, s);
    case 2: return launch_dt<2>(a, threads, smem, s);
    default: return launch_dt<4>(a, threads, smem, s);
    }
}

}  // namespace apax
