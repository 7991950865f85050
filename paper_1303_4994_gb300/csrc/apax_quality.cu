// apax_quality.cu -- the profiler's signal-quality metrics beyond the sums
// (Sec. 4): the 2-sigma S2R margin of window 4 and the spectral levels of
// window 3, for an array x and its decoded y.
//
// 2-sigma S2R margin.  The per-sample ratio |x| / |d|, d = x - y rounded
// once to binary64 (+inf where d = 0, 0 where x = 0 and d != 0), rounded
// once; the margin is the k-th smallest ratio, k = floor(45 n / 1000), so
// that 95.5% of the samples lie at or above it.  Non-negative binary64
// values order like their bit patterns, so the ratios' bits are radix-
// selected a byte at a time: one pass writes the keys and counts the top
// byte, then each of 8 steps picks the byte holding rank k (one CTA) and the
// next pass counts the following byte among the keys that match so far.
// The result is the exact order statistic: the same bits as a sort.
//
// Spectra.  Welch-Bartlett averages over full segments of L = 4096 samples
// (the largest power of two <= n below that): mean removed, periodic Hann
// window, |FFT|^2 / sum(w^2) in binary64, bins 1..L/2.  x and y share one
// complex FFT (x + i y, split by symmetry); d, real, packs its even and odd
// samples into one complex FFT of L/2 points (the real-input FFT by
// splitting: D[k] = E[k] + W^k O[k], E and O the half-length spectra of the
// even and odd samples, read off by the same symmetry).  A fixed number of
// CTAs (kSpecCtas, independent of the device) each add the periodograms of
// their segments in order; the bins' sums over the CTAs follow in CTA order,
// so the result does not depend on scheduling.  Peak = max, floor = lower
// median (sorted in shared memory), and the residual's mean level = the mean
// of 10 log10 P_d over the bins (added in a fixed tree).
#include <math.h>

#include "apax_device.cuh"
#include "apax_kernels.h"

namespace apax {

namespace {

constexpr int kSel = 256;        // radix-select buckets (a byte)
constexpr int kSpecL = 4096;     // segment length
// CTAs adding periodograms: fixed, so the sums are reproducible; one per SM
// of a GB300 (about 146 KB of shared memory each, so one CTA a SM), one wave
constexpr int kSpecCtas = 152;
constexpr int kSpecThreads = 512;


template <int DT>
__device__ __forceinline__ double as_double(const void *p, uint64_t i)
{
    if constexpr (DT == 1) return (double)reinterpret_cast<const int8_t *>(p)[i];
    else if constexpr (DT == 2) return (double)reinterpret_cast<const int16_t *>(p)[i];
    else if constexpr (DT == 3) return (double)reinterpret_cast<const int32_t *>(p)[i];
    else if constexpr (DT == 4) return (double)reinterpret_cast<const float *>(p)[i];
    else return reinterpret_cast<const double *>(p)[i];
}

template <int DT>
__global__ void k_s2r_keys(const void *x, const void *y, uint64_t n, unsigned long long *keys,
                           unsigned long long *hist)
{
    __shared__ unsigned int h[kSel];
    for (int i = threadIdx.x; i < kSel; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double xv = as_double<DT>(x, i), yv = as_double<DT>(y, i);
        const double d = fabs(__dsub_rn(xv, yv));
        const double r = d == 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : __ddiv_rn(fabs(xv), d);
        const unsigned long long key = (unsigned long long)__double_as_longlong(r);
        keys[i] = key;
        atomicAdd(&h[key >> 56], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSel; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Counts the byte at st->shift of the keys whose higher bytes equal the
// prefix.
__global__ void k_s2r_count(const unsigned long long *keys, uint64_t n, const SelState *st,
                            unsigned long long *hist)
{
    __shared__ unsigned int h[kSel];
    for (int i = threadIdx.x; i < kSel; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int sh = st->shift;
    const unsigned long long hi_mask = ~0ull << (sh + 8), want = st->prefix & hi_mask;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if ((key & hi_mask) == want) atomicAdd(&h[(key >> sh) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSel; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// One CTA: the bucket holding rank k, then the next byte (or the result).
__global__ void k_s2r_pick(SelState *st, unsigned long long *hist, apax_quality *q)
{
    __shared__ unsigned long long c[kSel];
    const int t = threadIdx.x;
    c[t] = hist[t];
    __syncthreads();
    if (t == 0) {
        unsigned long long k = st->k, acc = 0;
        int b = 0;
        for (; b < kSel - 1; ++b) {
            if (k < acc + c[b]) break;
            acc += c[b];
        }
        st->prefix |= (unsigned long long)b << st->shift;
        st->k = k - acc;
        if (st->shift == 0) q->s2r_ratio = __longlong_as_double((long long)st->prefix);
        st->shift -= 8;
    }
    hist[t] = 0;
}

// ---------------------------------------------------------------- spectra
// a b with one product of each part fused: re = fma(a.x, b.x, -(a.y b.y)),
// im = fma(a.x, b.y, a.y b.x) (four binary64 operations instead of six;
// the spectra are compared within a tolerance, not bit for bit)
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)),
                        __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}

// In-place radix-2 decimation-in-time FFT of z[0..L) (bit-reversed copy in,
// natural order out), twiddles exp(-2 pi i j / L) = tw[j << tws], j < L/2
// (tws = 1: a half-length transform reading the full table).  L is a power
// of two.  Stage s combines pairs half = 2^s apart, butterfly b at
// (b >> s) 2 half + (b & (half - 1)) with twiddle tw[pos L / (2 half)].
// Two stages run per pass over shared memory: a thread takes the four points
// of two stages' butterflies and does both in registers, the same operations
// on the same values as the stage-by-stage order, with half the barriers.
__device__ __forceinline__ void bfly(double2 &u, double2 &v, double2 w)
{
    const double2 t = cmul(v, w);
    const double2 a = u;
    u = make_double2(__dadd_rn(a.x, t.x), __dadd_rn(a.y, t.y));
    v = make_double2(__dsub_rn(a.x, t.x), __dsub_rn(a.y, t.y));
}

__device__ void fft_smem(double2 *z, const double2 *tw, int L, int logL, int tws)
{
    int stage = 0;
    for (; stage + 1 < logL; stage += 2) {
        const int half = 1 << stage;
        const int sh1 = logL - 1 - stage + tws, sh2 = logL - 2 - stage + tws;
        for (int b = threadIdx.x; b < L / 4; b += blockDim.x) {
            const int grp = b >> stage, pos = b & (half - 1);
            const int i0 = (grp << (stage + 2)) + pos;
            double2 p0 = z[i0], p1 = z[i0 + half], p2 = z[i0 + 2 * half], p3 = z[i0 + 3 * half];
            const double2 w1 = tw[pos << sh1];
            bfly(p0, p1, w1);  // stage s: (i0, i0 + half), (i0 + 2 half, i0 + 3 half)
            bfly(p2, p3, w1);
            bfly(p0, p2, tw[pos << sh2]);           // stage s + 1: pairs 2 half apart
            bfly(p1, p3, tw[(pos + half) << sh2]);
            z[i0] = p0;
            z[i0 + half] = p1;
            z[i0 + 2 * half] = p2;
            z[i0 + 3 * half] = p3;
        }
        __syncthreads();
    }
    if (stage < logL) {  // an odd number of stages: the last one alone
        const int half = 1 << stage;
        for (int b = threadIdx.x; b < L / 2; b += blockDim.x) {
            const int grp = b >> stage, pos = b & (half - 1);
            const int i0 = (grp << (stage + 1)) + pos;
            double2 p0 = z[i0], p1 = z[i0 + half];
            bfly(p0, p1, tw[pos << tws]);
            z[i0] = p0;
            z[i0 + half] = p1;
        }
        __syncthreads();
    }
}

// The periodic Hann window (1 - cos(2 pi m / L)) / 2 from the twiddles.
__device__ __forceinline__ double hann(const double2 *tw, int m, int H)
{
    const double c_ = m < H ? tw[m].x : -tw[m - H].x;
    return __dmul_rn(0.5, __dsub_rn(1.0, c_));
}

__device__ __forceinline__ int bitrev(int i, int logL) { return (int)(__brev((unsigned)i) >> (32 - logL)); }

// Fixed-order sum of v[0..m) across the CTA (m <= 2 blockDim): a tree over
// threads after each thread's sequential slice.
__device__ double cta_sum(double *buf, double mine)
{
    buf[threadIdx.x] = mine;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) buf[threadIdx.x] = __dadd_rn(buf[threadIdx.x], buf[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = buf[0];
    __syncthreads();
    return r;
}

__global__ void k_twiddles(double2 *tw, int L)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L / 2; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)L, &s, &c);
        tw[j] = make_double2(c, s);
    }
}

// CTA c adds the periodograms of segments c, c + gridDim.x, ... into
// part[c][3][L/2] (x, y, d; bins 1..L/2).
template <int DT>
__global__ void __launch_bounds__(kSpecThreads) k_spectra(const void *x, const void *y, int L,
                                                         int logL, uint64_t segs,
                                                         const double2 *tw_g, double *part)
{
    extern __shared__ double2 sm[];
    double2 *z = sm;                 // L complex
    double2 *tw = sm + L;            // L/2 twiddles
    double *acc = reinterpret_cast<double *>(tw + L / 2);  // 3 * L/2
    double *red = acc + 3 * (L / 2);                      // blockDim.x
    const int H = L / 2;
    for (int j = threadIdx.x; j < H; j += blockDim.x) tw[j] = tw_g[j];
    for (int j = threadIdx.x; j < 3 * H; j += blockDim.x) acc[j] = 0.0;
    __syncthreads();
    // sum of the periodic Hann window's squares: 3L/8 exactly
    const double wnorm = 3.0 * (double)L / 8.0;
    const int logL_ = logL;
    for (uint64_t s = blockIdx.x; s < segs; s += gridDim.x) {
        const uint64_t base = s * (uint64_t)L;
        // means of x, y, d over the segment
        double sx = 0.0, sy = 0.0, sd = 0.0;
        for (int m = threadIdx.x; m < L; m += blockDim.x) {
            const double xv = as_double<DT>(x, base + m), yv = as_double<DT>(y, base + m);
            sx = __dadd_rn(sx, xv);
            sy = __dadd_rn(sy, yv);
            sd = __dadd_rn(sd, __dsub_rn(xv, yv));
        }
        const double mx = cta_sum(red, sx) / L, my = cta_sum(red, sy) / L, md = cta_sum(red, sd) / L;
        // x and y: z = w (x - mx) + i w (y - my), one L-point FFT
        for (int m = threadIdx.x; m < L; m += blockDim.x) {
            const double xv = as_double<DT>(x, base + m), yv = as_double<DT>(y, base + m);
            const double w = hann(tw, m, H);
            z[bitrev(m, logL_)] = make_double2(__dmul_rn(w, __dsub_rn(xv, mx)), __dmul_rn(w, __dsub_rn(yv, my)));
        }
        __syncthreads();
        fft_smem(z, tw, L, logL_, 0);
        for (int k = 1 + threadIdx.x; k <= H; k += blockDim.x) {
            const double2 a = z[k], b = z[(L - k) & (L - 1)];
            // X = (Z[k] + conj Z[L-k]) / 2, Y = (Z[k] - conj Z[L-k]) / (2i)
            const double xr = 0.5 * __dadd_rn(a.x, b.x), xi = 0.5 * __dsub_rn(a.y, b.y);
            const double yr = 0.5 * __dadd_rn(a.y, b.y), yi = -0.5 * __dsub_rn(a.x, b.x);
            acc[k - 1] = __dadd_rn(acc[k - 1], __dadd_rn(__dmul_rn(xr, xr), __dmul_rn(xi, xi)) / wnorm);
            acc[H + k - 1] = __dadd_rn(acc[H + k - 1], __dadd_rn(__dmul_rn(yr, yr), __dmul_rn(yi, yi)) / wnorm);
        }
        __syncthreads();
        // d: v = w (d - md); z[m] = v[2m] + i v[2m+1], one L/2-point FFT
        for (int m = threadIdx.x; m < H; m += blockDim.x) {
            double v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int mm = 2 * m + e;
                const double xv = as_double<DT>(x, base + mm), yv = as_double<DT>(y, base + mm);
                v[e] = __dmul_rn(hann(tw, mm, H), __dsub_rn(__dsub_rn(xv, yv), md));
            }
            z[bitrev(m, logL_ - 1)] = make_double2(v[0], v[1]);
        }
        __syncthreads();
        fft_smem(z, tw, H, logL_ - 1, 1);
        for (int k = 1 + threadIdx.x; k <= H; k += blockDim.x) {
            double dr, di;
            if (k < H) {
                // E = (Z[k] + conj Z[H-k]) / 2, O = (Z[k] - conj Z[H-k]) / (2i), D = E + W^k O
                const double2 a = z[k], b = z[H - k];
                const double er = 0.5 * __dadd_rn(a.x, b.x), ei = 0.5 * __dsub_rn(a.y, b.y);
                const double orr = 0.5 * __dadd_rn(a.y, b.y), oi = -0.5 * __dsub_rn(a.x, b.x);
                const double2 t = cmul(make_double2(orr, oi), tw[k]);
                dr = __dadd_rn(er, t.x);
                di = __dadd_rn(ei, t.y);
            } else {
                // D[L/2] = E[0] - O[0], both real
                dr = __dsub_rn(z[0].x, z[0].y);
                di = 0.0;
            }
            acc[2 * H + k - 1] = __dadd_rn(acc[2 * H + k - 1], __dadd_rn(__dmul_rn(dr, dr), __dmul_rn(di, di)) / wnorm);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < 3 * H; j += blockDim.x) part[(uint64_t)blockIdx.x * 3 * H + j] = acc[j];
}

// P[j] = (sum over CTAs, in CTA order, of part[c][j]) / segs.
__global__ void k_spec_bins(const double *part, int ctas, int m, uint64_t segs, double *P)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s = __dadd_rn(s, part[(uint64_t)c * m + j]);
    P[j] = s / (double)segs;
}

// One CTA (1024 threads): sort each of the three spectra (H <= 2048 values)
// in shared memory, take max and lower median, and the mean of 10 log10 P_d.
__global__ void __launch_bounds__(1024) k_spec_stats(const double *P, int H, apax_quality *q)
{
    __shared__ double v[2048];
    __shared__ double red[1024];
    double peak[3], flo[3];
    for (int a = 0; a < 3; ++a) {
        for (int j = threadIdx.x; j < 2048; j += blockDim.x)
            v[j] = j < H ? P[a * H + j] : __longlong_as_double(0x7ff0000000000000ll);
        __syncthreads();
        // bitonic sort of 2048 values
        for (int size = 2; size <= 2048; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int j = threadIdx.x; j < 1024; j += blockDim.x) {
                    const int lo = 2 * j - (j & (stride - 1)), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const double a0 = v[lo], a1 = v[hi];
                    if ((a0 > a1) == up) {
                        v[lo] = a1;
                        v[hi] = a0;
                    }
                }
                __syncthreads();
            }
        }
        peak[a] = v[H - 1];
        flo[a] = v[(H - 1) / 2];
        __syncthreads();
    }
    // mean of 10 log10 P_d (fixed tree)
    double s = 0.0;
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        const double p = P[2 * H + j];
        s = __dadd_rn(s, p > 0.0 ? 10.0 * log10(p) : __longlong_as_double(0xfff0000000000000ll));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        q->peak_x = peak[0];
        q->floor_x = flo[0];
        q->peak_y = peak[1];
        q->floor_y = flo[1];
        q->peak_d = peak[2];
        q->floor_d = flo[2];
        q->mean_d_db = red[0] / (double)H;
    }
}

__global__ void k_s2r_init(SelState *st, unsigned long long k)
{
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->k = k;
        st->shift = 56;
    }
}

template <int DT>
cudaError_t quality_dt(const QualityArgs &a, cudaStream_t s)
{
    const int sms = sm_count();
    const uint64_t want = (a.n + 255) / 256, cap = (uint64_t)sms * 8;
    const unsigned grid = (unsigned)(a.n ? (want < cap ? want : cap) : 1);
    if (a.n) {
        k_s2r_init<<<1, 32, 0, s>>>(a.state, (45ull * a.n) / 1000ull);
        k_s2r_keys<DT><<<grid, 256, 0, s>>>(a.x, a.y, a.n, a.keys, a.hist);
        for (int step = 0; step < 8; ++step) {
            k_s2r_pick<<<1, kSel, 0, s>>>(a.state, a.hist, a.q);
            if (step < 7) k_s2r_count<<<grid, 256, 0, s>>>(a.keys, a.n, a.state, a.hist);
        }
    }
    if (a.segs) {
        k_twiddles<<<8, 256, 0, s>>>(a.tw, a.L);
        const int H = a.L / 2;
        const size_t smem = (size_t)a.L * 16 + (size_t)H * 16 + (size_t)3 * H * 8 + kSpecThreads * 8;
        cudaError_t e = smem_limit<k_spectra<DT>>(smem);
        if (e != cudaSuccess) return e;
        const int ctas = (int)quality_spectral_ctas(a.segs);
        k_spectra<DT><<<ctas, kSpecThreads, smem, s>>>(a.x, a.y, a.L, a.logL, a.segs, a.tw, a.part);
        k_spec_bins<<<(3 * H + 255) / 256, 256, 0, s>>>(a.part, ctas, 3 * H, a.segs, a.P);
        k_spec_stats<<<1, 1024, 0, s>>>(a.P, H, a.q);
    }
    return cudaGetLastError();
}

}  // namespace

uint64_t quality_spectral_ctas(uint64_t segs) { return segs < (uint64_t)kSpecCtas ? segs : kSpecCtas; }

namespace {
__global__ void k_quality_header(apax_quality *q, apax_quality h)
{
    if (threadIdx.x == 0) *q = h;
}
}  // namespace

cudaError_t launch_quality_header(apax_quality *q, const apax_quality &h, cudaStream_t s)
{
    k_quality_header<<<1, 32, 0, s>>>(q, h);
    return cudaGetLastError();
}

cudaError_t launch_quality(const QualityArgs &a, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return quality_dt<1>(a, s);
    case 2: return quality_dt<2>(a, s);
    case 3: return quality_dt<3>(a, s);
    case 4: return quality_dt<4>(a, s);
    default: return quality_dt<5>(a, s);
    }
}

}  // namespace apax
