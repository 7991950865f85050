/*
 * apax_oracle.c -- CPU oracle of the APAX block encoder, decoder and profiler.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, scalar restatement of the
 * method of Wegener, "Universal Numerical Encoder and Profiler Reduces
 * Computing's Memory Wall with Software, FPGA, and SoC Implementations"
 * (arXiv 1303.4994), in the frozen reading of the bitstream that the CUDA
 * library also implements.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Every routine follows one passage of the paper:
 *   Sec. 6, block diagram paragraph: blocks of 64..16384 samples (multiple
 *       of 4); attenuator multiplying each sample by a per-block value;
 *       redundancy remover choosing among the data and its filtered versions;
 *       the best-stream decision of block j carried in block j+1's header;
 *       a 4-byte (integer) or 6-byte (float) block header.
 *   Sec. 6, bit-packer paragraph: block floating point with one exponent per
 *       group of 4 samples (or, in the second container version, of 8),
 *       joint exponent encoding (nine 4-bit joint tokens, five 4-bit single
 *       tokens, 8-bit absolute tokens, the first exponent of a block
 *       absolute).
 *   Sec. 5: derivatives remove sample-to-sample redundancy (Fig. 3b); the
 *       signal monitor's correlated-neighbour choice adds, in the second
 *       container version, the sum of neighbours for near-Nyquist data.
 *   Sec. 4: profiler -- rate/correlation sweep, r = sum(xy)/sqrt(sum x^2 sum y^2),
 *       recommended operating point at a correlation target.
 * Where the paper is silent the reading is stated beside the code; the
 * complete list of readings is kept with the design notes of the project.
 *
 * Parity pins (tests/test_oracle_pins.py): the hand-derived worked example,
 * the closed-form fixed-rate size, lossless round trip at code 0 for
 * integers, exhaustive JEE token round trips, rounding against exact
 * rationals, exact metric sums against rational arithmetic, and the
 * fixed-rate search against exhaustive search on tiny blocks.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <float.h>

/* Status codes of the C interface (same numeric contract as the library). */
#define ST_OK            0
#define ST_INVALID_ARG  -1
#define ST_BLOCK_SIZE   -2
#define ST_DTYPE        -3
#define ST_RATE         -4
#define ST_CAPACITY     -5
#define ST_TOO_LARGE    -6
#define ST_NONFINITE    -8
#define ST_CORRUPT      -9

enum { DT_I8 = 1, DT_I16 = 2, DT_I32 = 3, DT_F32 = 4, DT_F64 = 5 };
enum { MODE_FR = 0, MODE_FQ = 1 };
/* Format options (container version 2): BFPE groups of 8 samples (Sec. 6
 * bit packer, "groups of 4 or 8"); the sum stream u_i = q_i + q_{i-1} as a
 * fourth choice of the redundancy remover (Sec. 6 signal monitor, Sec. 5
 * Fig. 3b: data near the Nyquist frequency alternate in sign). */
enum { FMT_GROUP8 = 1, FMT_SUM_STREAM = 2, FMT_ALL = 3 };

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Format description of one array                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dtype;
    int size;      /* bytes per element */
    int width;     /* W: integer domain width (Sec. 6 readings: 8/16/32, floats 32) */
    int isfloat;
    int Q;         /* float quantiser precision: 23 (f32), 29 (f64) */
    int hbits;     /* block header bits: 32 (ints), 48 (floats) -- Sec. 6 */
    uint32_t N;    /* block size */
    int fmt;       /* format options (FMT_*) */
    int gs;        /* BFPE group size: 4, or 8 with FMT_GROUP8 */
    int nstreams;  /* streams the redundancy remover compares: 3, or 4 with FMT_SUM_STREAM */
} fmt_t;

static int fmt_init(fmt_t *f, int dtype, uint32_t N, int fmt)
{
    memset(f, 0, sizeof *f);
    f->dtype = dtype;
    f->N = N;
    if (fmt & ~FMT_ALL) return ST_INVALID_ARG;
    f->fmt = fmt;
    f->gs = (fmt & FMT_GROUP8) ? 8 : 4;
    f->nstreams = (fmt & FMT_SUM_STREAM) ? 4 : 3;
    switch (dtype) {
    case DT_I8:  f->size = 1; f->width = 8;  break;
    case DT_I16: f->size = 2; f->width = 16; break;
    case DT_I32: f->size = 4; f->width = 32; break;
    case DT_F32: f->size = 4; f->width = 32; f->isfloat = 1; f->Q = 23; break;
    case DT_F64: f->size = 8; f->width = 32; f->isfloat = 1; f->Q = 29; break;
    default: return ST_DTYPE;
    }
    f->hbits = f->isfloat ? 48 : 32;
    /* Sec. 6: "block size between 64 and 16,384 (any multiple of 4)"; with
     * groups of 8 the block holds whole groups (a multiple of 8). */
    if (N < 64 || N > 16384 || (N % (uint32_t)f->gs) != 0) return ST_BLOCK_SIZE;
    return ST_OK;
}

static int64_t read_int(const void *x, int dtype, uint64_t i)
{
    switch (dtype) {
    case DT_I8:  return ((const int8_t *)x)[i];
    case DT_I16: return ((const int16_t *)x)[i];
    default:     return ((const int32_t *)x)[i];
    }
}

static double read_flt(const void *x, int dtype, uint64_t i)
{
    if (dtype == DT_F32) return (double)((const float *)x)[i];
    return ((const double *)x)[i];
}

/* ------------------------------------------------------------------------ */
/* Exact integer helpers                                                     */
/* ------------------------------------------------------------------------ */

/* Round-half-to-even of t / 2^s for integer t (exact rational rounding).
 * s <= 0 multiplies by 2^-s (caller guarantees it fits). */
static i128 rne_div_pow2(i128 t, int s)
{
    if (s <= 0) return t * ((i128)1 << (-s));
    if (s > 124) return 0; /* |t| < 2^123 everywhere this is used */
    i128 q = t >> s; /* floor division (arithmetic shift) */
    i128 r = t - q * ((i128)1 << s);       /* 0 <= r < 2^s */
    i128 half = (i128)1 << (s - 1);
    if (r > half || (r == half && (q & 1))) q += 1;
    return q;
}

/* Reduce v modulo 2^W into the signed W-bit range (two's complement). */
static int32_t wrap_w(int64_t v, int W)
{
    uint64_t m = (W >= 32) ? 0xffffffffull : ((1ull << W) - 1);
    uint64_t u = (uint64_t)v & m;
    if ((u >> (W - 1)) & 1) return (int32_t)((int64_t)u - (int64_t)(m + 1));
    return (int32_t)u;
}

/* bits(v): number of bits of the two's-complement representation of v
 * (0 for v == 0): least b with -2^(b-1) <= v <= 2^(b-1)-1.  Sec. 6 BFPE
 * "exponent that indicates the number of bits in each of the next N samples". */
static int bits_of(int32_t v)
{
    if (v == 0) return 0;
    for (int b = 1; b <= 32; ++b) {
        int64_t lo = -((int64_t)1 << (b - 1));
        int64_t hi = ((int64_t)1 << (b - 1)) - 1;
        if (v >= lo && v <= hi) return b;
    }
    return 32;
}

/* ------------------------------------------------------------------------ */
/* Attenuation code (Sec. 6 attenuator)                                      */
/* ------------------------------------------------------------------------ */
/* Reading: 12-bit code c, k = c >> 7, m = c & 127, a(c) = (256-m) 2^-(8+k);
 * the top code 4095 is the zero attenuator a = 0. */
static void code_split(int c, int *k, int *m)
{
    *k = c >> 7;
    *m = c & 127;
}

/* Reciprocal table of the decoder: R[m] = RNE(2^32 / (256 - m)). */
static int64_t recip_R(int m)
{
    i128 num = (i128)1 << 32;
    i128 d = 256 - m;
    i128 q = num / d, r = num - q * d;
    if (2 * r > d || (2 * r == d && (q & 1))) q += 1;
    return (int64_t)q;
}

/* ------------------------------------------------------------------------ */
/* Quantiser (attenuator output) and dequantiser                             */
/* ------------------------------------------------------------------------ */

/* Exponent E_b of a float block: max|x| = f 2^E_b, f in [0.5, 1); 0 for an
 * all-zero block.  Returns ST_NONFINITE if any sample is NaN or infinite. */
static int block_exponent(const fmt_t *F, const void *x, uint64_t off, int L, int *Eb)
{
    double mx = 0.0;
    for (int i = 0; i < L; ++i) {
        double v = read_flt(x, F->dtype, off + i);
        if (!isfinite(v)) return ST_NONFINITE;
        double a = fabs(v);
        if (a > mx) mx = a;
    }
    int e = 0;
    if (mx != 0.0) (void)frexp(mx, &e);
    *Eb = e;
    return ST_OK;
}

/* q = RNE(x a(c)) for integers; q = RNE(x 2^(Q-E_b) a(c)) for floats, the
 * exact real product rounded once. */
static int32_t quantise_value(const fmt_t *F, const void *x, uint64_t i, int c, int Eb)
{
    if (c == 4095) return 0;
    int k, m;
    code_split(c, &k, &m);
    if (!F->isfloat) {
        i128 t = (i128)read_int(x, F->dtype, i) * (256 - m);
        return (int32_t)rne_div_pow2(t, 8 + k);
    }
    double v = read_flt(x, F->dtype, i);
    if (v == 0.0) return 0;
    int e;
    double f = frexp(fabs(v), &e);          /* |v| = f 2^e, f in [0.5,1) */
    int64_t M = (int64_t)ldexp(f, 53);      /* integer significand (exact) */
    int ex = e - 53;                         /* |v| = M 2^ex */
    i128 P = (i128)M * (256 - m);
    /* |v| 2^(Q-Eb) (256-m) 2^-(8+k) = P 2^(Q - Eb + ex - 8 - k) */
    int sh = (8 + k) - (F->Q - Eb + ex);
    i128 q = rne_div_pow2(P, sh);
    return (int32_t)(v < 0 ? -q : q);
}

/* Round the exact value V 2^e to binary32 or binary64 (ties to even),
 * saturating at the largest finite magnitude. */
static double round_to_format(i128 V, int e, int isf64)
{
    if (V == 0) return 0.0;
    int neg = V < 0;
    u128 A = neg ? (u128)(-V) : (u128)V;
    int p = isf64 ? 53 : 24, emin = isf64 ? -1022 : -126, emax = isf64 ? 1023 : 127;
    int nb = 0;
    for (u128 t = A; t; t >>= 1) ++nb;
    int top = e + nb - 1;                       /* value in [2^top, 2^(top+1)) */
    int u = top - (p - 1);                      /* exponent of the last kept bit */
    if (u < emin - (p - 1)) u = emin - (p - 1); /* subnormal grid */
    i128 mant = rne_div_pow2((i128)A, u - e);   /* exact when u <= e */
    /* mant <= 2^p and the value is mant 2^u; saturate beyond the format */
    int mb = 0;
    for (i128 t = mant; t; t >>= 1) ++mb;
    double r;
    if (mb > 0 && u + mb - 1 > emax)
        r = isf64 ? DBL_MAX : (double)FLT_MAX;
    else
        r = ldexp((double)mant, u);
    return neg ? -r : r;
}

/* Stores V (integers: clamped to the type) or RN(V 2^e) (floats) into y[i]. */
static void store_value(const fmt_t *F, void *y, uint64_t i, i128 V, int e)
{
    if (!F->isfloat) {
        int64_t lo, hi;
        switch (F->dtype) {
        case DT_I8:  lo = INT8_MIN;  hi = INT8_MAX;  break;
        case DT_I16: lo = INT16_MIN; hi = INT16_MAX; break;
        default:     lo = INT32_MIN; hi = INT32_MAX; break;
        }
        i128 v = V;
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        switch (F->dtype) {
        case DT_I8:  ((int8_t *)y)[i] = (int8_t)v;  break;
        case DT_I16: ((int16_t *)y)[i] = (int16_t)v; break;
        default:     ((int32_t *)y)[i] = (int32_t)v; break;
        }
        return;
    }
    double r = round_to_format(V, e, F->dtype == DT_F64);
    if (F->dtype == DT_F32) ((float *)y)[i] = (float)r;
    else ((double *)y)[i] = r;
}

/* Decoder arithmetic: y = q R[m] 2^(k-24) for integers (rounded to nearest
 * even, clamped); y = RN(q R[m] 2^(E_b - Q + k - 24)) for floats. */
static void dequantise_value(const fmt_t *F, int32_t q, int c, int Eb, void *y, uint64_t i)
{
    if (c == 4095 || q == 0) { store_value(F, y, i, 0, 0); return; }
    int k, m;
    code_split(c, &k, &m);
    i128 V = (i128)q * recip_R(m);
    if (!F->isfloat) {
        i128 r = (k <= 23) ? rne_div_pow2(V, 24 - k) : V * ((i128)1 << (k - 24));
        store_value(F, y, i, r, 0);
    } else {
        store_value(F, y, i, V, Eb - F->Q + k - 24);
    }
}

/* ------------------------------------------------------------------------ */
/* Redundancy remover, exponents, JEE tokens                                 */
/* ------------------------------------------------------------------------ */

/* Streams (Sec. 5/6: the data and selected derivatives), within the block,
 * modulo 2^W:  S0 u_i = q_i;  S1 u_0 = q_0, u_i = q_i - q_{i-1};
 * S2 u_0 = q_0, u_1 = q_1 - q_0, u_i = q_i - 2 q_{i-1} + q_{i-2};
 * S3 (sum stream) u_0 = q_0, u_i = q_i + q_{i-1}. */
static void derive_stream(const int32_t *q, int len, int s, int W, int32_t *u)
{
    for (int i = 0; i < len; ++i) {
        int64_t v;
        if (s == 0 || i == 0) v = q[i];
        else if (s == 3) v = (int64_t)q[i] + q[i - 1];
        else if (s == 1 || i == 1) v = (int64_t)q[i] - q[i - 1];
        else v = (int64_t)q[i] - 2 * (int64_t)q[i - 1] + q[i - 2];
        u[i] = wrap_w(v, W);
    }
}

/* Group exponent (BFPE, groups of gs = 4 or 8): largest bits() of the
 * group; a width of 31 is promoted to 32 so that every exponent fits the
 * 5-bit absolute field. */
static void group_exponents(const int32_t *u, int G, int gs, int *e)
{
    for (int g = 0; g < G; ++g) {
        int b = 0;
        for (int j = 0; j < gs; ++j) {
            int t = bits_of(u[gs * g + j]);
            if (t > b) b = t;
        }
        e[g] = (b == 31) ? 32 : b;
    }
}

static int iabs_(int v) { return v < 0 ? -v : v; }

/* JEE (Sec. 6): the first exponent is absolute; then, greedily left to right,
 * two successive diffs both in [-1,1] make one joint nibble 3(d1+1)+(d2+1)
 * (codes 0..8); a diff in [-2,2] that cannot pair makes a single nibble
 * 11+d (codes 9..13); any other exponent is absolute: nibble 14+(v>>4) then
 * nibble v&15 with v = min(e, 31) (v = 31 stands for 32).  Returns the count. */
static int jee_encode(const int *e, int G, uint8_t *nib)
{
    int t = 0;
    int v = e[0] >= 31 ? 31 : e[0];
    nib[t++] = (uint8_t)(14 + (v >> 4));
    nib[t++] = (uint8_t)(v & 15);
    int i = 1;
    while (i <= G - 1) {
        int d = e[i] - e[i - 1];
        if (i + 1 <= G - 1) {
            int d2 = e[i + 1] - e[i];
            if (iabs_(d) <= 1 && iabs_(d2) <= 1) {
                nib[t++] = (uint8_t)(3 * (d + 1) + (d2 + 1));
                i += 2;
                continue;
            }
        }
        if (iabs_(d) <= 2) {
            nib[t++] = (uint8_t)(11 + d);
        } else {
            v = e[i] >= 31 ? 31 : e[i];
            nib[t++] = (uint8_t)(14 + (v >> 4));
            nib[t++] = (uint8_t)(v & 15);
        }
        i += 1;
    }
    return t;
}

/* Inverse of jee_encode: reads nibbles until G exponents are known.  Returns
 * the nibble count, or -1 if the stream is malformed or longer than maxnib. */
static int jee_decode(const uint8_t *nib, int maxnib, int G, int W, int *e)
{
    int t = 0, g = 0;
    while (g < G) {
        if (t >= maxnib) return -1;
        int a = nib[t++];
        if (a >= 14) {
            if (t >= maxnib) return -1;
            int v = ((a - 14) << 4) | nib[t++];
            if (v > 31) return -1;
            e[g++] = (v == 31) ? 32 : v;
        } else {
            if (g == 0) return -1; /* first exponent must be absolute */
            if (a <= 8) {
                if (g + 1 >= G) return -1; /* a joint token needs two diffs */
                int d1 = a / 3 - 1, d2 = a % 3 - 1;
                e[g] = e[g - 1] + d1; ++g;
                e[g] = e[g - 1] + d2; ++g;
            } else {
                e[g] = e[g - 1] + (a - 11); ++g;
            }
        }
    }
    for (int i = 0; i < G; ++i) {
        int lim = (W >= 32) ? 32 : W;
        if (e[i] < 0 || e[i] > lim || e[i] == 31) return -1;
    }
    return t;
}

/* ------------------------------------------------------------------------ */
/* Bit writer / reader: LSB-first bit strings in little-endian bytes         */
/* ------------------------------------------------------------------------ */
typedef struct { uint8_t *buf; uint64_t bit; } bitw_t;

static void put_bits(bitw_t *w, uint64_t v, int n)
{
    for (int i = 0; i < n; ++i) {
        if ((v >> i) & 1) w->buf[w->bit >> 3] |= (uint8_t)(1u << (w->bit & 7));
        w->bit++;
    }
}

typedef struct { const uint8_t *buf; uint64_t bit, end; } bitr_t;

static int get_bits(bitr_t *r, int n, uint64_t *out)
{
    uint64_t v = 0;
    if (r->bit + (uint64_t)n > r->end) return -1;
    for (int i = 0; i < n; ++i) {
        if ((r->buf[r->bit >> 3] >> (r->bit & 7)) & 1) v |= (uint64_t)1 << i;
        r->bit++;
    }
    *out = v;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One block                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L, G;        /* samples and groups of this block */
    int Eb;          /* float block exponent (0 for ints) */
    int32_t q[16384];
    int32_t u[16384];
    int e[4096];
    uint8_t nib[8192];
    int nnib;
} blk_t;

/* Quantise block j at code c: q[0..gs G), the tail replicating q[L-1]. */
static int quantise_block(const fmt_t *F, const void *x, uint64_t n, uint64_t j, int c, blk_t *b)
{
    uint64_t off = j * F->N;
    uint64_t rem = n - off;
    b->L = (int)(rem < F->N ? rem : F->N);
    b->G = (b->L + F->gs - 1) / F->gs;
    b->Eb = 0;
    if (F->isfloat) {
        int st = block_exponent(F, x, off, b->L, &b->Eb);
        if (st) return st;
    }
    for (int i = 0; i < b->L; ++i) b->q[i] = quantise_value(F, x, off + i, c, b->Eb);
    for (int i = b->L; i < F->gs * b->G; ++i) b->q[i] = b->q[b->L - 1];
    return ST_OK;
}

/* Unpadded packet bits of the quantised block b with stream s. */
static uint64_t packet_bits(const fmt_t *F, blk_t *b, int s)
{
    derive_stream(b->q, F->gs * b->G, s, F->width, b->u);
    group_exponents(b->u, b->G, F->gs, b->e);
    b->nnib = jee_encode(b->e, b->G, b->nib);
    uint64_t bits = (uint64_t)F->hbits + 4u * (uint64_t)b->nnib;
    for (int g = 0; g < b->G; ++g) bits += (uint64_t)F->gs * (uint64_t)b->e[g];
    return bits;
}

static uint64_t pad32_bytes(uint64_t bits) { return 4 * ((bits + 31) / 32); }

/* best(j): the stream with the fewest packet bits at code 0 (ties to the
 * lower index) among S0..S2, and S3 with the sum-stream option.  Sec. 6: the
 * redundancy remover keeps whichever candidate stream packs into the fewest
 * bits; the signal monitor's say over which neighbours are correlated is
 * read as offering the sum stream, which the same fewest-bits rule takes
 * exactly when it is the smallest. */
static int best_stream(const fmt_t *F, const void *x, uint64_t n, uint64_t j, blk_t *b, int *st)
{
    *st = quantise_block(F, x, n, j, 0, b);
    if (*st) return 0;
    int best = 0;
    uint64_t bb = packet_bits(F, b, 0);
    for (int s = 1; s < F->nstreams; ++s) {
        uint64_t t = packet_bits(F, b, s);
        if (t < bb) { bb = t; best = s; }
    }
    return best;
}

/* Writes the packet of the quantised block (stream s, code c) into out,
 * padded with zeros to plen bytes; plen is stored in the header. */
static void write_packet(const fmt_t *F, blk_t *b, int s, int c, uint8_t *out, uint64_t plen)
{
    (void)packet_bits(F, b, s);
    memset(out, 0, plen);
    bitw_t w = { out, 0 };
    put_bits(&w, (uint64_t)s, 2);
    put_bits(&w, (uint64_t)c, 12);
    put_bits(&w, plen, 18);
    if (F->isfloat) put_bits(&w, (uint64_t)(uint16_t)(int16_t)b->Eb, 16);
    for (int t = 0; t < b->nnib; ++t) put_bits(&w, b->nib[t], 4);
    for (int g = 0; g < b->G; ++g)
        for (int i = 0; i < F->gs; ++i) {
            int e = b->e[g];
            uint64_t v = (uint64_t)(uint32_t)b->u[F->gs * g + i];
            if (e < 64) v &= (e == 0) ? 0 : (((uint64_t)1 << e) - 1);
            put_bits(&w, v, e);
        }
}

/* ------------------------------------------------------------------------ */
/* Fixed-rate budgets (reading of the adaptive loop's packet-size target)    */
/* ------------------------------------------------------------------------ */
static uint64_t min_packet(const fmt_t *F, int L)
{
    int G = (L + F->gs - 1) / F->gs;
    uint64_t bits = (uint64_t)F->hbits + 8 + 4 * (uint64_t)((G - 1 + 1) / 2);
    return pad32_bytes(bits);
}

static uint64_t fr_budget(const fmt_t *F, int L, uint32_t num, uint32_t den)
{
    uint64_t b = ((uint64_t)L * F->size * den / (4ull * num)) * 4;
    uint64_t mp = min_packet(F, L);
    return b > mp ? b : mp;
}

/* ------------------------------------------------------------------------ */
/* Container (40-byte header) helpers                                        */
/* ------------------------------------------------------------------------ */
static void put_le(uint8_t *p, uint64_t v, int nbytes)
{
    for (int i = 0; i < nbytes; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_le(const uint8_t *p, int nbytes)
{
    uint64_t v = 0;
    for (int i = 0; i < nbytes; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

static uint64_t nblocks_of(uint64_t n, uint32_t N) { return (n + N - 1) / N; }

static uint64_t table_bytes(uint64_t nb) { return ((4 * nb) + 7) / 8 * 8; }

static int check_params(const fmt_t *F, int mode, uint32_t num, uint32_t den, int c)
{
    if (mode == MODE_FR) {
        if (num == 0 || den == 0) return ST_RATE;
        uint64_t B = ((uint64_t)F->N * F->size * den / (4ull * num)) * 4;
        if (B < min_packet(F, (int)F->N)) return ST_RATE;
        if (B >= (1u << 18)) return ST_RATE;
    } else if (mode == MODE_FQ) {
        if (c < 0 || c > 4095) return ST_INVALID_ARG;
    } else {
        return ST_INVALID_ARG;
    }
    return ST_OK;
}

/* ------------------------------------------------------------------------ */
/* Exported: sizes                                                           */
/* ------------------------------------------------------------------------ */

/* Fixed rate: the exact size; fixed quality: the worst-case bound. */
int oracle_encoded_size(int dtype, uint64_t n, uint32_t N, int fmt, int mode, uint32_t num,
                        uint32_t den, int c, uint64_t *bytes)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    st = check_params(&F, mode, num, den, c);
    if (st) return st;
    uint64_t nb = nblocks_of(n, N);
    if (nb == 0) { *bytes = 40; return ST_OK; }
    uint64_t Lend = n - (nb - 1) * N;
    if (mode == MODE_FR) {
        uint64_t B = fr_budget(&F, (int)N, num, den);
        *bytes = 40 + (nb - 1) * B + fr_budget(&F, (int)Lend, num, den);
    } else {
        uint64_t wmax = (uint64_t)F.width;
        uint64_t full = pad32_bytes((uint64_t)F.hbits + 8ull * (N / F.gs) + wmax * N);
        int Gl = (int)((Lend + F.gs - 1) / F.gs);
        uint64_t last = pad32_bytes((uint64_t)F.hbits + 8ull * Gl + wmax * (uint64_t)F.gs * Gl);
        *bytes = 40 + table_bytes(nb) + (nb - 1) * full + last;
    }
    return ST_OK;
}

/* Fixed-rate budget B of a full block and minimum packet (for tests). */
int oracle_fr_budget(int dtype, uint32_t N, int fmt, int L, uint32_t num, uint32_t den,
                     uint64_t *B)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    *B = fr_budget(&F, L, num, den);
    return ST_OK;
}

int oracle_min_packet(int dtype, uint32_t N, int fmt, int L, uint64_t *bytes)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    *bytes = min_packet(&F, L);
    return ST_OK;
}

/* ------------------------------------------------------------------------ */
/* Exported: encoder                                                         */
/* ------------------------------------------------------------------------ */

/* The 40-byte container header (reading 11): magic "APX1", version (1; 2
 * when a format option is on), dtype, mode, flags (bit 0: offset table;
 * bit 1: groups of 8; bit 2: sum stream), N, the fixed-quality code, the
 * fixed-rate budget B, n; the payload size at bytes 28..35 is written once
 * the packets are placed. */
static void write_container_header(uint8_t *out, const fmt_t *F, int mode, int cfq,
                                   uint64_t B, uint64_t n)
{
    memset(out, 0, 40);
    out[0] = 'A'; out[1] = 'P'; out[2] = 'X'; out[3] = '1';
    out[4] = F->fmt ? 2 : 1;
    out[5] = (uint8_t)F->dtype;
    out[6] = (uint8_t)mode;
    out[7] = (uint8_t)(((mode == MODE_FQ) ? 1 : 0) | (F->fmt << 1));
    const uint32_t N = F->N;
    put_le(out + 8, N, 4);
    put_le(out + 12, mode == MODE_FQ ? (uint64_t)cfq : 0, 2);
    put_le(out + 16, B, 4);
    put_le(out + 20, n, 8);
}


/* Fixed-rate search (reading of the adaptive loop, policy BISECT): c = 0 if
 * it fits; else bisection on [0, 4095] keeping hi fitting (4095 always fits). */
static int fr_bisect(const fmt_t *F, const void *x, uint64_t n, uint64_t j, int s,
                     uint64_t budget, blk_t *b, int *st)
{
    *st = quantise_block(F, x, n, j, 0, b);
    if (*st) return 0;
    if (pad32_bytes(packet_bits(F, b, s)) <= budget) return 0;
    int lo = 0, hi = 4095;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        *st = quantise_block(F, x, n, j, mid, b);
        if (*st) return 0;
        if (pad32_bytes(packet_bits(F, b, s)) <= budget) hi = mid;
        else lo = mid;
    }
    return hi;
}

/* Fixed-rate search, policy PREDICT (the adaptive loop of Sec. 6 read as a
 * prediction from the code-0 packet, then a short walk up a ladder of codes).
 * Attenuating by 2^-k narrows every group of exponent e by min(e, k) bits,
 * so red(k) = gs sum_g min(e_g, k) bits are predicted to go (gs samples per
 * group); with the excess
 * D = packet_bits(0) - 8 B_j, k1 is the least k in 1..31 with red(k) >= D
 * (31 if none), and the fraction f = ceil(16 (D - red(k1-1)) /
 * (red(k1) - red(k1-1))) clamped to 1..16 (16 if the denominator is 0)
 * places the start between the power-of-two codes 128(k1-1) and 128 k1:
 * c = 128(k1-1) + M[f] for f < 16, else 128 k1, where a(128 k + M[f]) is
 * 2^-(k + f/16) rounded to the attenuator's 8-bit grid,
 * M[f] = RNE(256 (1 - 2^(-f/16))).  From there c climbs the ladder of codes
 * 128 k + M[f'] (k = 0..31, f' = 0..15, then 4095, which always fits) until
 * the packet fits.  As with BISECT, c = 0 when the code-0 packet already
 * fits. */
static const int ladder_M[16] = { 0, 11, 21, 31, 41, 50, 59, 67, 75, 83, 90, 97, 104, 110, 116, 122 };

static int ladder_next(int c)
{
    int k = c >> 7, m = c & 127;
    for (int f = 0; f < 16; ++f)
        if (ladder_M[f] > m) return 128 * k + ladder_M[f];
    return k < 31 ? 128 * (k + 1) : 4095;
}

static int fr_predict(const fmt_t *F, const void *x, uint64_t n, uint64_t j, int s,
                      uint64_t budget, blk_t *b, int *st)
{
    *st = quantise_block(F, x, n, j, 0, b);
    if (*st) return 0;
    uint64_t bits0 = packet_bits(F, b, s); /* also leaves the code-0 exponents in b->e */
    if (pad32_bytes(bits0) <= budget) return 0;
    int64_t D = (int64_t)bits0 - 8 * (int64_t)budget;
    int64_t red[32];
    red[0] = 0;
    for (int k = 1; k < 32; ++k) {
        int64_t r = 0;
        for (int g = 0; g < b->G; ++g) r += F->gs * (int64_t)(b->e[g] < k ? b->e[g] : k);
        red[k] = r;
    }
    int k1 = 31;
    for (int k = 1; k < 32; ++k)
        if (red[k] >= D) { k1 = k; break; }
    int64_t num = 16 * (D - red[k1 - 1]), den = red[k1] - red[k1 - 1];
    int64_t f;
    if (den == 0) {
        f = 16;
    } else {
        f = num / den; /* truncation toward zero, then the ceiling */
        if (f * den < num) f += 1;
    }
    if (f < 1) f = 1;
    if (f > 16) f = 16;
    int c = f < 16 ? 128 * (k1 - 1) + ladder_M[f] : 128 * k1;
    for (;;) {
        *st = quantise_block(F, x, n, j, c, b);
        if (*st) return 0;
        if (c >= 4095 || pad32_bytes(packet_bits(F, b, s)) <= budget) return c;
        c = ladder_next(c);
    }
}

enum { SEARCH_BISECT = 0, SEARCH_PREDICT = 1 };

static int fr_search(const fmt_t *F, const void *x, uint64_t n, uint64_t j, int s,
                     uint64_t budget, blk_t *b, int *st, int search)
{
    return search == SEARCH_PREDICT ? fr_predict(F, x, n, j, s, budget, b, st)
                                    : fr_bisect(F, x, n, j, s, budget, b, st);
}

int oracle_encode_s(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, int mode,
                    uint32_t num, uint32_t den, int cfq, int search, uint8_t *out, uint64_t cap,
                    uint64_t *bytes)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    st = check_params(&F, mode, num, den, cfq);
    if (st) return st;
    uint64_t nb = nblocks_of(n, N);
    if (cap < 40) return ST_CAPACITY;
    uint64_t B = (mode == MODE_FR) ? fr_budget(&F, (int)N, num, den) : 0;
    write_container_header(out, &F, mode, cfq, B, n);

    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    if (!b) return ST_INVALID_ARG;
    uint64_t payload_off = 40 + ((mode == MODE_FQ) ? table_bytes(nb) : 0);
    if (payload_off > cap) { free(b); return ST_CAPACITY; }
    if (mode == MODE_FQ) memset(out + 40, 0, payload_off - 40);
    uint64_t pos = 0; /* payload bytes written */
    int prev_best = 0;
    for (uint64_t j = 0; j < nb; ++j) {
        int bj = best_stream(&F, x, n, j, b, &st);
        if (st) { free(b); return st; }
        int s = (j == 0) ? bj : prev_best;
        prev_best = bj;
        int c;
        uint64_t plen;
        if (mode == MODE_FQ) {
            c = cfq;
            st = quantise_block(&F, x, n, j, c, b);
            if (st) { free(b); return st; }
            plen = pad32_bytes(packet_bits(&F, b, s));
        } else {
            int L = (int)((n - j * N) < N ? (n - j * N) : N);
            uint64_t budget = fr_budget(&F, L, num, den);
            c = fr_search(&F, x, n, j, s, budget, b, &st, search);
            if (st) { free(b); return st; }
            st = quantise_block(&F, x, n, j, c, b);
            if (st) { free(b); return st; }
            plen = budget;
        }
        if (mode == MODE_FQ) {
            if (pos / 4 > 0xffffffffull) { free(b); return ST_TOO_LARGE; }
            put_le(out + 40 + 4 * j, pos / 4, 4);
        }
        if (payload_off + pos + plen > cap) { free(b); return ST_CAPACITY; }
        write_packet(&F, b, s, c, out + payload_off + pos, plen);
        pos += plen;
    }
    free(b);
    put_le(out + 28, pos, 8);
    *bytes = payload_off + pos;
    return ST_OK;
}

int oracle_encode(const void *x, int dtype, uint64_t n, uint32_t N, int mode, uint32_t num,
                  uint32_t den, int cfq, uint8_t *out, uint64_t cap, uint64_t *bytes)
{
    return oracle_encode_s(x, dtype, n, N, 0, mode, num, den, cfq, SEARCH_BISECT, out, cap, bytes);
}

/* ------------------------------------------------------------------------ */
/* Exported: decoder                                                         */
/* ------------------------------------------------------------------------ */

/* Decodes one packet starting at p (at most avail bytes) into y[off..off+L). */
static int decode_packet(const fmt_t *F, const uint8_t *p, uint64_t avail, int L, void *y,
                         uint64_t off, uint64_t *plen_out, blk_t *b)
{
    bitr_t r = { p, 0, 8 * avail };
    uint64_t v;
    if (get_bits(&r, 2, &v)) return ST_CORRUPT;
    int s = (int)v;
    if (s >= F->nstreams) return ST_CORRUPT; /* S3 only with the sum-stream option */
    if (get_bits(&r, 12, &v)) return ST_CORRUPT;
    int c = (int)v;
    if (get_bits(&r, 18, &v)) return ST_CORRUPT;
    uint64_t plen = v;
    if (plen < 4 || (plen % 4) != 0 || plen > avail) return ST_CORRUPT;
    r.end = 8 * plen;
    int Eb = 0;
    if (F->isfloat) {
        if (get_bits(&r, 16, &v)) return ST_CORRUPT;
        Eb = (int16_t)(uint16_t)v;
    }
    const int gs = F->gs;
    int G = (L + gs - 1) / gs;
    /* token section: read nibbles lazily through a small buffer */
    int maxnib = (int)((r.end - r.bit) / 4);
    if (maxnib > 2 * G) maxnib = 2 * G;
    for (int t = 0; t < maxnib; ++t) {
        uint64_t nv;
        bitr_t rr = r;
        rr.bit = r.bit + 4ull * t;
        if (get_bits(&rr, 4, &nv)) return ST_CORRUPT;
        b->nib[t] = (uint8_t)nv;
    }
    int nn = jee_decode(b->nib, maxnib, G, F->width, b->e);
    if (nn < 0) return ST_CORRUPT;
    r.bit += 4ull * nn;
    for (int g = 0; g < G; ++g)
        for (int i = 0; i < gs; ++i) {
            int e = b->e[g];
            uint64_t m = 0;
            if (e > 0 && get_bits(&r, e, &m)) return ST_CORRUPT;
            int64_t sv = 0;
            if (e > 0) {
                sv = (int64_t)m;
                if ((m >> (e - 1)) & 1) sv -= (int64_t)1 << e;
            }
            b->u[gs * g + i] = wrap_w(sv, F->width);
        }
    /* inverse streams, modulo 2^W */
    int ng = gs * G;
    for (int i = 0; i < ng; ++i) {
        int64_t qv;
        if (s == 0 || i == 0) qv = b->u[i];
        else if (s == 3) qv = (int64_t)b->u[i] - b->q[i - 1];
        else if (s == 1 || i == 1) qv = (int64_t)b->u[i] + b->q[i - 1];
        else qv = (int64_t)b->u[i] + 2 * (int64_t)b->q[i - 1] - b->q[i - 2];
        b->q[i] = wrap_w(qv, F->width);
    }
    for (int i = 0; i < L; ++i) dequantise_value(F, b->q[i], c, Eb, y, off + i);
    *plen_out = plen;
    return ST_OK;
}

/* Parsed container header (reading 11). */
typedef struct {
    fmt_t F;
    int mode;
    uint64_t B, payload, nb, poff;
} cont_t;

static int parse_container(const uint8_t *in, uint64_t in_bytes, int dtype, uint64_t n, cont_t *c)
{
    if (in_bytes < 40) return ST_CORRUPT;
    if (in[0] != 'A' || in[1] != 'P' || in[2] != 'X' || in[3] != '1') return ST_CORRUPT;
    /* version 1: no format option; version 2: at least one (flags bits 1-2) */
    const int fmt = (in[7] >> 1) & 0x7f;
    if (!((in[4] == 1 && fmt == 0) || (in[4] == 2 && fmt != 0 && fmt <= FMT_ALL)))
        return ST_CORRUPT;
    if (in[5] != dtype) return ST_INVALID_ARG;
    c->mode = in[6];
    uint32_t N = (uint32_t)get_le(in + 8, 4);
    uint64_t hn = get_le(in + 20, 8);
    if (hn != n) return ST_INVALID_ARG;
    if (fmt_init(&c->F, dtype, N, fmt)) return ST_CORRUPT;
    if (c->mode != MODE_FR && c->mode != MODE_FQ) return ST_CORRUPT;
    c->B = get_le(in + 16, 4);
    c->payload = get_le(in + 28, 8);
    c->nb = nblocks_of(n, N);
    c->poff = 40 + ((c->mode == MODE_FQ) ? table_bytes(c->nb) : 0);
    if (c->poff > in_bytes || c->payload > in_bytes - c->poff) return ST_CORRUPT;
    return ST_OK;
}

/* Decodes blocks [b0, b1) of a parsed container into y (at their places). */
static int decode_range(const cont_t *c, const uint8_t *in, void *y, uint64_t n, uint64_t b0,
                        uint64_t b1, blk_t *b)
{
    const uint32_t N = c->F.N;
    for (uint64_t j = b0; j < b1; ++j) {
        uint64_t start = (c->mode == MODE_FQ) ? 4 * get_le(in + 40 + 4 * j, 4) : j * c->B;
        if (start >= c->payload) return ST_CORRUPT;
        int L = (int)((n - j * N) < N ? (n - j * N) : N);
        uint64_t plen;
        int st = decode_packet(&c->F, in + c->poff + start, c->payload - start, L, y, j * N,
                               &plen, b);
        if (st) return st;
        if (c->mode == MODE_FR && j + 1 < c->nb && plen != c->B) return ST_CORRUPT;
    }
    return ST_OK;
}

int oracle_decode(const uint8_t *in, uint64_t in_bytes, void *y, int dtype, uint64_t n)
{
    cont_t c;
    int st = parse_container(in, in_bytes, dtype, n, &c);
    if (st) return st;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    if (!b) return ST_INVALID_ARG;
    st = decode_range(&c, in, y, n, 0, c.nb, b);
    free(b);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Exact sums (profiler metrics)                                             */
/* ------------------------------------------------------------------------ */
/* Reading of the metric arithmetic (Sec. 4 gives only the formula): each
 * block's sums of x, y, x^2, xy, y^2 and d^2 (d = x - y) are formed exactly
 * and rounded once to binary64; the array totals are binary64 sums of the
 * block values in a fixed fan-in-16 tree (runs of 16 consecutive values added
 * left to right, level after level). */

#define SA_LO (-2304)
#define SA_ND 160
typedef struct { int64_t d[SA_ND]; } sacc_t;

/* a += sign * v * 2^e (v < 2^107) */
static void sa_add(sacc_t *a, int neg, u128 v, int e)
{
    if (v == 0) return;
    int p = e - SA_LO;
    int di = p >> 5, sh = p & 31;
    for (int i = 0; i < 4; ++i) {
        uint64_t chunk = (uint64_t)(v >> (32 * i)) & 0xffffffffull;
        if (!chunk) continue;
        uint64_t t = chunk << sh;
        int64_t lo = (int64_t)(t & 0xffffffffull), hi = (int64_t)(t >> 32);
        if (neg) { lo = -lo; hi = -hi; }
        a->d[di + i] += lo;
        a->d[di + i + 1] += hi;
    }
}

static double sa_round(const sacc_t *a)
{
    uint32_t w[SA_ND + 1];
    int64_t carry = 0;
    for (int i = 0; i < SA_ND; ++i) {
        int64_t t = a->d[i] + carry;
        uint32_t low = (uint32_t)((uint64_t)t & 0xffffffffull);
        carry = (t - (int64_t)low) / ((int64_t)1 << 32);
        w[i] = low;
    }
    int neg = carry < 0;
    if (neg) { /* two's complement negate */
        uint64_t c = 1;
        for (int i = 0; i < SA_ND; ++i) {
            uint64_t t = (uint64_t)(uint32_t)~w[i] + c;
            w[i] = (uint32_t)t;
            c = t >> 32;
        }
    }
    int top = -1;
    for (int i = SA_ND - 1; i >= 0; --i) if (w[i]) { top = i; break; }
    if (top < 0) return 0.0;
    int hb = 31;
    while (!((w[top] >> hb) & 1)) --hb;
    int topbit = 32 * top + hb;                 /* bit index of the leading one */
    int texp = topbit + SA_LO;                  /* exponent of the leading one */
    int u = texp - 52;
    if (u < -1074) u = -1074;
    int ubit = u - SA_LO;                       /* bit index of the unit to keep */
    /* mant = bits [ubit, topbit]; round on the rest */
    u128 mant = 0;
    for (int bi = topbit; bi >= ubit; --bi)
        mant = (mant << 1) | ((w[bi >> 5] >> (bi & 31)) & 1);
    int half = 0, sticky = 0;
    if (ubit >= 1) {
        int hb1 = ubit - 1;
        half = (w[hb1 >> 5] >> (hb1 & 31)) & 1;
        /* sticky: any one bit strictly below hb1 */
        int wi = hb1 >> 5, bi = hb1 & 31;
        if (bi > 0 && (w[wi] & ((1u << bi) - 1))) sticky = 1;
        for (int t = wi - 1; t >= 0 && !sticky; --t)
            if (w[t]) sticky = 1;
    }
    if (half && (sticky || (mant & 1))) mant += 1;
    double r = ldexp((double)mant, u);
    return neg ? -r : r;
}

/* Exact value of element i as (sign, integer significand, exponent). */
static void split_value(const fmt_t *F, const void *v, uint64_t i, int *neg, u128 *M, int *e)
{
    if (!F->isfloat) {
        int64_t t = read_int(v, F->dtype, i);
        *neg = t < 0;
        *M = (u128)(t < 0 ? -(i128)t : (i128)t);
        *e = 0;
        return;
    }
    double t = read_flt(v, F->dtype, i);
    *neg = t < 0;
    if (t == 0.0) { *M = 0; *e = 0; return; }
    int ex;
    double f = frexp(fabs(t), &ex);
    *M = (u128)(uint64_t)ldexp(f, 53);
    *e = ex - 53;
}

/* Block sums of one block: out[0..5] = x, y, x^2, xy, y^2, d^2. */
static void block_sums(const fmt_t *F, const void *x, const void *y, uint64_t off, int L, double *out)
{
    sacc_t *S = (sacc_t *)calloc(6, sizeof(sacc_t));
    for (int i = 0; i < L; ++i) {
        int nx, ny, ex, ey;
        u128 mx, my;
        split_value(F, x, off + i, &nx, &mx, &ex);
        split_value(F, y, off + i, &ny, &my, &ey);
        sa_add(&S[0], nx, mx, ex);
        sa_add(&S[1], ny, my, ey);
        sa_add(&S[2], 0, mx * mx, 2 * ex);
        sa_add(&S[3], nx ^ ny, mx * my, ex + ey);
        sa_add(&S[4], 0, my * my, 2 * ey);
        /* (x - y)^2 = x^2 - 2xy + y^2, exactly */
        sa_add(&S[5], 0, mx * mx, 2 * ex);
        sa_add(&S[5], !(nx ^ ny), mx * my, ex + ey + 1);
        sa_add(&S[5], 0, my * my, 2 * ey);
    }
    for (int k = 0; k < 6; ++k) out[k] = sa_round(&S[k]);
    free(S);
}

static double tree16(double *v, uint64_t cnt)
{
    if (cnt == 0) return 0.0;
    while (cnt > 1) {
        uint64_t m = (cnt + 15) / 16;
        for (uint64_t j = 0; j < m; ++j) {
            double s = v[16 * j];
            for (uint64_t i = 1; i < 16 && 16 * j + i < cnt; ++i) s += v[16 * j + i];
            v[j] = s;
        }
        cnt = m;
    }
    return v[0];
}

/* Per-block sums (6 per block, block-major) for blocks [b0, b1). */
int oracle_block_sums(const void *x, const void *y, int dtype, uint64_t n, uint32_t N,
                      uint64_t b0, uint64_t b1, double *out)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, 0); /* the sums do not depend on the packet format */
    if (st) return st;
    for (uint64_t j = b0; j < b1; ++j) {
        uint64_t off = j * N;
        int L = (int)((n - off) < N ? (n - off) : N);
        block_sums(&F, x, y, off, L, out + 6 * (j - b0));
    }
    return ST_OK;
}

/* Totals: out[0..5] = sum x, sum y, sum x^2, sum xy, sum y^2, sum d^2. */
int oracle_metrics(const void *x, const void *y, int dtype, uint64_t n, uint32_t N, double *out)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, 0);
    if (st) return st;
    uint64_t nb = nblocks_of(n, N);
    double *bs = (double *)malloc(sizeof(double) * 6 * (nb ? nb : 1));
    double *col = (double *)malloc(sizeof(double) * (nb ? nb : 1));
    st = oracle_block_sums(x, y, dtype, n, N, 0, nb, bs);
    for (int k = 0; k < 6; ++k) {
        for (uint64_t j = 0; j < nb; ++j) col[j] = bs[6 * j + k];
        out[k] = tree16(col, nb);
    }
    free(bs);
    free(col);
    return st;
}

/* r = sum(xy) / sqrt(sum(x^2) sum(y^2)), the Sec. 4 formula in binary64. */
double oracle_corr(double sxx, double sxy, double syy)
{
    /* sums beyond binary64 give a quiet NaN with a fixed bit pattern */
    if (!isfinite(sxx) || !isfinite(sxy) || !isfinite(syy)) {
        uint64_t b = 0x7ff8000000000000ull;
        double r;
        memcpy(&r, &b, sizeof r);
        return r;
    }
    if (sxx == 0.0 && syy == 0.0) return 1.0;
    if (sxx == 0.0 || syy == 0.0) return 0.0;
    double p = sxx * syy;
    if (isfinite(p) && p >= DBL_MIN) return sxy / sqrt(p);
    return (sxy / sqrt(sxx)) / sqrt(syy);
}

/* ------------------------------------------------------------------------ */
/* Exported: profiler                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t code;
    uint32_t flags;
    uint64_t bytes;         /* fixed-quality container size at this code */
    double sx, sy, sxx, sxy, syy, sdd;
    double r;
} oracle_point;

/* Sec. 4: for each candidate code, encode (fixed quality) and decode the
 * array, then compare the decoded y with the original x.  Candidates are any
 * strictly increasing codes of 0..4095 (Sec. 6: the attenuator's
 * multiplier is a floating-point value, not only a power of two).  The
 * recommended
 * point is the largest i with r_j >= target for all j <= i (candidates in
 * increasing attenuation); 0 if even r_0 misses the target. */
int oracle_profile(const void *x, int dtype, uint64_t n, uint32_t N, int fmt,
                   const uint16_t *cand, int ncand, double target, oracle_point *pts,
                   int *recommended)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    if (ncand < 1) return ST_INVALID_ARG;
    for (int i = 0; i < ncand; ++i) {
        if (cand[i] > 4095) return ST_INVALID_ARG;
        if (i > 0 && cand[i] <= cand[i - 1]) return ST_INVALID_ARG;
    }
    uint64_t cap;
    st = oracle_encoded_size(dtype, n, N, fmt, MODE_FQ, 1, 1, 0, &cap);
    if (st) return st;
    uint8_t *buf = (uint8_t *)malloc(cap);
    void *y = malloc((size_t)(n ? n : 1) * F.size);
    int rec = -1, ok_prefix = 1;
    for (int i = 0; i < ncand; ++i) {
        uint64_t bytes;
        st = oracle_encode_s(x, dtype, n, N, fmt, MODE_FQ, 1, 1, cand[i], SEARCH_BISECT, buf,
                             cap, &bytes);
        if (st) break;
        st = oracle_decode(buf, bytes, y, dtype, n);
        if (st) break;
        double s[6];
        oracle_metrics(x, y, dtype, n, N, s);
        pts[i].code = cand[i];
        pts[i].flags = 0;
        pts[i].bytes = bytes;
        pts[i].sx = s[0]; pts[i].sy = s[1]; pts[i].sxx = s[2];
        pts[i].sxy = s[3]; pts[i].syy = s[4]; pts[i].sdd = s[5];
        pts[i].r = oracle_corr(s[2], s[3], s[4]);
        if (ok_prefix && pts[i].r >= target) rec = i;
        else ok_prefix = 0;
    }
    free(buf);
    free(y);
    if (st) return st;
    *recommended = rec < 0 ? 0 : rec;
    return rec < 0 ? 1 : ST_OK; /* 1: even the first candidate misses the target */
}

/* ------------------------------------------------------------------------ */
/* Exported helpers for the parity pins                                      */
/* ------------------------------------------------------------------------ */
int oracle_bits(int32_t v) { return bits_of(v); }

int64_t oracle_recip(int m) { return recip_R(m); }

int64_t oracle_rne_shift(int64_t t, int s) { return (int64_t)rne_div_pow2(t, s); }

int oracle_jee_encode(const int *e, int G, uint8_t *nib) { return jee_encode(e, G, nib); }

int oracle_jee_decode(const uint8_t *nib, int maxnib, int G, int *e)
{
    return jee_decode(nib, maxnib, G, 32, e);
}

/* Quantise one value of a block whose exponent is Eb (Eb ignored for ints). */
int32_t oracle_quantise(const void *x, int dtype, uint64_t i, int c, int Eb)
{
    fmt_t F;
    if (fmt_init(&F, dtype, 64, 0)) return 0;
    return quantise_value(&F, x, i, c, Eb);
}

/* Dequantise one value into y[0]. */
int oracle_dequantise(int32_t q, int dtype, int c, int Eb, void *y)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, 64, 0);
    if (st) return st;
    dequantise_value(&F, q, c, Eb, y, 0);
    return ST_OK;
}

int oracle_block_exponent(const void *x, int dtype, uint64_t off, int L, int *Eb)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, 64, 0);
    if (st) return st;
    return block_exponent(&F, x, off, L, Eb);
}

/* Unpadded packet bits of block j at code c with stream s (tests). */
int oracle_packet_bits(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, uint64_t j,
                       int c, int s, uint64_t *bits)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    st = quantise_block(&F, x, n, j, c, b);
    if (!st) *bits = packet_bits(&F, b, s);
    free(b);
    return st;
}

/* Streams chosen for blocks [b0, b1) (the one-block lag of Sec. 6). */
int oracle_streams(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, uint64_t b0,
                   uint64_t b1, int *streams)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    for (uint64_t j = b0; j < b1; ++j) {
        uint64_t pj = j == 0 ? 0 : j - 1;
        streams[j - b0] = best_stream(&F, x, n, pj, b, &st);
        if (st) break;
    }
    free(b);
    return st;
}

/* Fixed-rate code that the search picks for block j given stream s. */
int oracle_fr_code(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, uint64_t j,
                   int s, uint64_t budget, int search, int *code)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    *code = fr_search(&F, x, n, j, s, budget, b, &st, search);
    free(b);
    return st;
}

/* Packets of blocks [b0, b1) of an array encoded with the given parameters,
 * written back to back into out (for sampled parity at full size).  For
 * fixed rate, the packets are padded to their budgets; for fixed quality to
 * 32 bits.  lens[j-b0] receives each packet length. */
int oracle_encode_blocks(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, int mode,
                         uint32_t num, uint32_t den, int cfq, int search, uint64_t b0,
                         uint64_t b1, uint8_t *out, uint64_t cap, uint64_t *lens)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    st = check_params(&F, mode, num, den, cfq);
    if (st) return st;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    uint64_t pos = 0;
    for (uint64_t j = b0; j < b1; ++j) {
        int s = best_stream(&F, x, n, j == 0 ? 0 : j - 1, b, &st);
        if (st) break;
        int L = (int)((n - j * N) < N ? (n - j * N) : N);
        int c;
        uint64_t plen;
        if (mode == MODE_FQ) {
            c = cfq;
            st = quantise_block(&F, x, n, j, c, b);
            if (st) break;
            plen = pad32_bytes(packet_bits(&F, b, s));
        } else {
            uint64_t budget = fr_budget(&F, L, num, den);
            c = fr_search(&F, x, n, j, s, budget, b, &st, search);
            if (st) break;
            st = quantise_block(&F, x, n, j, c, b);
            if (st) break;
            plen = budget;
        }
        if (pos + plen > cap) { st = ST_CAPACITY; break; }
        write_packet(&F, b, s, c, out + pos, plen);
        lens[j - b0] = plen;
        pos += plen;
    }
    free(b);
    return st;
}

/* Derived profiler metrics (Sec. 4, Window 2) from the six sums and the
 * sample count n: out = [r, r_centred, snr_db, rms_pct, rms_db, mean_x,
 * mean_y, mean_d, std_x, std_y, std_d].  r is the printed uncentred formula;
 * r_centred is the textbook Pearson coefficient; snr_db = 10 log10(sum x^2 /
 * sum d^2); rms_pct = 100 sqrt(sum d^2 / sum x^2); rms_db = 20 log10(rms_pct /
 * 100) (the Table 3 relation between its two RMS columns); standard
 * deviations are population deviations. */
int oracle_derived(const double *s, uint64_t n, double *out)
{
    double sx = s[0], sy = s[1], sxx = s[2], sxy = s[3], syy = s[4], sdd = s[5];
    double nn = (double)n;
    out[0] = oracle_corr(sxx, sxy, syy);
    if (n == 0) {
        for (int i = 1; i < 11; ++i) out[i] = 0.0;
        return ST_OK;
    }
    double vx = sxx - sx * sx / nn, vy = syy - sy * sy / nn, cv = sxy - sx * sy / nn;
    if (vx <= 0.0 && vy <= 0.0) out[1] = 1.0;
    else if (vx <= 0.0 || vy <= 0.0) out[1] = 0.0;
    else out[1] = cv / sqrt(vx * vy);
    if (sdd == 0.0) {
        out[2] = INFINITY;
        out[3] = 0.0;
        out[4] = -INFINITY;
    } else if (sxx == 0.0) {
        out[2] = -INFINITY;
        out[3] = INFINITY;
        out[4] = INFINITY;
    } else {
        out[2] = 10.0 * log10(sxx / sdd);
        out[3] = 100.0 * sqrt(sdd / sxx);
        out[4] = 20.0 * log10(out[3] / 100.0);
    }
    double mx = sx / nn, my = sy / nn, md = (sx - sy) / nn;
    out[5] = mx;
    out[6] = my;
    out[7] = md;
    double t;
    t = sxx / nn - mx * mx; out[8] = sqrt(t > 0.0 ? t : 0.0);
    t = syy / nn - my * my; out[9] = sqrt(t > 0.0 ? t : 0.0);
    t = sdd / nn - md * md; out[10] = sqrt(t > 0.0 ? t : 0.0);
    return ST_OK;
}

/* ------------------------------------------------------------------------ */
/* Threaded drivers over contiguous block ranges                             */
/* ------------------------------------------------------------------------ */
/* The same per-block routines as above (oracle_encode_blocks for the
 * packets, decode_range for decoding, block_sums for the metrics), run by
 * POSIX threads on contiguous ranges of blocks; the container, the decoded
 * array and the sums are identical to the single-threaded calls because
 * every block is coded on its own (Sec. 6; the one-block lag only reads the
 * predecessor block's samples) and the ranges are assembled in block order.
 * They exist so that whole arrays of benchmark size can be checked and timed
 * on all host cores.  threads <= 0 means one per online core. */
#include <pthread.h>
#include <unistd.h>

static int mt_threads(int threads, uint64_t nb)
{
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > nb) threads = nb ? (int)nb : 1;
    return threads;
}

int oracle_threads(int threads) { return mt_threads(threads, (uint64_t)1 << 40); }

typedef struct {
    /* encode */
    const void *x;
    int dtype, fmt, mode, cfq, search;
    uint64_t n;
    uint32_t N, num, den;
    uint64_t b0, b1;
    uint8_t *buf;
    uint64_t cap;
    uint64_t *lens;
    /* decode */
    const cont_t *c;
    const uint8_t *in;
    void *y;
    /* block sums */
    const void *yy;
    double *sums;
    int st;
} mt_job;

static void *enc_worker(void *p)
{
    mt_job *J = (mt_job *)p;
    J->st = oracle_encode_blocks(J->x, J->dtype, J->n, J->N, J->fmt, J->mode, J->num, J->den,
                                 J->cfq, J->search, J->b0, J->b1, J->buf, J->cap, J->lens);
    return NULL;
}

static void *dec_worker(void *p)
{
    mt_job *J = (mt_job *)p;
    blk_t *b = (blk_t *)malloc(sizeof(blk_t));
    J->st = b ? decode_range(J->c, J->in, J->y, J->n, J->b0, J->b1, b) : ST_INVALID_ARG;
    free(b);
    return NULL;
}

static void *sums_worker(void *p)
{
    mt_job *J = (mt_job *)p;
    J->st = oracle_block_sums(J->x, J->yy, J->dtype, J->n, J->N, J->b0, J->b1, J->sums);
    return NULL;
}

/* Runs fn on T jobs (the first in the calling thread); returns the status of
 * the lowest-numbered failing range, as the sequential loop would. */
static int mt_run(mt_job *jobs, int T, void *(*fn)(void *))
{
    pthread_t tid[256];
    int started[256];
    for (int i = 1; i < T; ++i) started[i] = pthread_create(&tid[i], NULL, fn, &jobs[i]) == 0;
    fn(&jobs[0]);
    for (int i = 1; i < T; ++i) {
        if (started[i]) pthread_join(tid[i], NULL);
        else fn(&jobs[i]);
    }
    for (int i = 0; i < T; ++i)
        if (jobs[i].st) return jobs[i].st;
    return ST_OK;
}

static void mt_split(mt_job *jobs, int T, uint64_t nb)
{
    for (int i = 0; i < T; ++i) {
        jobs[i].b0 = nb * (uint64_t)i / (uint64_t)T;
        jobs[i].b1 = nb * (uint64_t)(i + 1) / (uint64_t)T;
        jobs[i].st = ST_OK;
    }
}

/* oracle_encode, block ranges on `threads` threads. */
int oracle_encode_mt(const void *x, int dtype, uint64_t n, uint32_t N, int fmt, int mode,
                     uint32_t num, uint32_t den, int cfq, int search, uint8_t *out, uint64_t cap,
                     uint64_t *bytes, int threads)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    st = check_params(&F, mode, num, den, cfq);
    if (st) return st;
    const uint64_t nb = nblocks_of(n, N);
    if (cap < 40) return ST_CAPACITY;
    const uint64_t B = (mode == MODE_FR) ? fr_budget(&F, (int)N, num, den) : 0;
    write_container_header(out, &F, mode, cfq, B, n);
    const uint64_t payload_off = 40 + ((mode == MODE_FQ) ? table_bytes(nb) : 0);
    if (payload_off > cap) return ST_CAPACITY;
    if (mode == MODE_FQ) memset(out + 40, 0, payload_off - 40);
    const int T = mt_threads(threads, nb);
    /* largest packet of one block: the budget, or every exponent absolute at
     * the full width (the worst case the size bound also uses) */
    const uint64_t maxp = mode == MODE_FR
                              ? fr_budget(&F, (int)N, num, den)
                              : pad32_bytes((uint64_t)F.hbits + 8ull * (N / F.gs) + (uint64_t)F.width * N);
    mt_job jobs[256];
    memset(jobs, 0, sizeof jobs);
    mt_split(jobs, T, nb);
    uint64_t *lens = (uint64_t *)malloc(sizeof(uint64_t) * (nb ? nb : 1));
    int fail = lens == NULL;
    for (int i = 0; i < T && !fail; ++i) {
        mt_job *J = &jobs[i];
        J->x = x; J->dtype = dtype; J->fmt = fmt; J->n = n; J->N = N; J->mode = mode;
        J->num = num; J->den = den; J->cfq = cfq; J->search = search;
        J->cap = maxp * (J->b1 - J->b0);
        /* the last block's fixed-rate budget may exceed B (minimum packet) */
        if (mode == MODE_FR && J->b1 == nb && nb) {
            int L = (int)(n - (nb - 1) * N);
            uint64_t bl = fr_budget(&F, L, num, den);
            if (bl > maxp) J->cap += bl - maxp;
        }
        J->buf = (uint8_t *)malloc(J->cap ? J->cap : 1);
        J->lens = lens + J->b0;
        if (!J->buf) fail = 1;
    }
    if (fail) {
        for (int i = 0; i < T; ++i) free(jobs[i].buf);
        free(lens);
        return ST_INVALID_ARG;
    }
    st = mt_run(jobs, T, enc_worker);
    uint64_t pos = 0;
    for (int i = 0; i < T && !st; ++i) {
        const mt_job *J = &jobs[i];
        uint64_t q = 0;
        for (uint64_t j = J->b0; j < J->b1; ++j) {
            if (mode == MODE_FQ) {
                if ((pos + q) / 4 > 0xffffffffull) { st = ST_TOO_LARGE; break; }
                put_le(out + 40 + 4 * j, (pos + q) / 4, 4);
            }
            q += lens[j];
        }
        if (st) break;
        if (payload_off + pos + q > cap) { st = ST_CAPACITY; break; }
        memcpy(out + payload_off + pos, J->buf, q);
        pos += q;
    }
    for (int i = 0; i < T; ++i) free(jobs[i].buf);
    free(lens);
    if (st) return st;
    put_le(out + 28, pos, 8);
    *bytes = payload_off + pos;
    return ST_OK;
}

/* oracle_decode, block ranges on `threads` threads. */
int oracle_decode_mt(const uint8_t *in, uint64_t in_bytes, void *y, int dtype, uint64_t n,
                     int threads)
{
    cont_t c;
    int st = parse_container(in, in_bytes, dtype, n, &c);
    if (st) return st;
    const int T = mt_threads(threads, c.nb);
    mt_job jobs[256];
    memset(jobs, 0, sizeof jobs);
    mt_split(jobs, T, c.nb);
    for (int i = 0; i < T; ++i) {
        jobs[i].c = &c;
        jobs[i].in = in;
        jobs[i].y = y;
        jobs[i].n = n;
    }
    return mt_run(jobs, T, dec_worker);
}

/* oracle_metrics, the block sums on `threads` threads (the fan-in-16 tree
 * over the block values is the same sequential loop). */
int oracle_metrics_mt(const void *x, const void *y, int dtype, uint64_t n, uint32_t N,
                      double *out, int threads)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, 0);
    if (st) return st;
    const uint64_t nb = nblocks_of(n, N);
    double *bs = (double *)malloc(sizeof(double) * 6 * (nb ? nb : 1));
    double *col = (double *)malloc(sizeof(double) * (nb ? nb : 1));
    if (!bs || !col) {
        free(bs);
        free(col);
        return ST_INVALID_ARG;
    }
    const int T = mt_threads(threads, nb);
    mt_job jobs[256];
    memset(jobs, 0, sizeof jobs);
    mt_split(jobs, T, nb);
    for (int i = 0; i < T; ++i) {
        jobs[i].x = x;
        jobs[i].yy = y;
        jobs[i].dtype = dtype;
        jobs[i].n = n;
        jobs[i].N = N;
        jobs[i].sums = bs + 6 * jobs[i].b0;
    }
    st = mt_run(jobs, T, sums_worker);
    for (int k = 0; k < 6 && !st; ++k) {
        for (uint64_t j = 0; j < nb; ++j) col[j] = bs[6 * j + k];
        out[k] = tree16(col, nb);
    }
    free(bs);
    free(col);
    return st;
}

/* oracle_profile with the threaded encode, decode and sums. */
int oracle_profile_mt(const void *x, int dtype, uint64_t n, uint32_t N, int fmt,
                      const uint16_t *cand, int ncand, double target, oracle_point *pts,
                      int *recommended, int threads)
{
    fmt_t F;
    int st = fmt_init(&F, dtype, N, fmt);
    if (st) return st;
    if (ncand < 1) return ST_INVALID_ARG;
    for (int i = 0; i < ncand; ++i) {
        if (cand[i] > 4095) return ST_INVALID_ARG;
        if (i > 0 && cand[i] <= cand[i - 1]) return ST_INVALID_ARG;
    }
    uint64_t cap;
    st = oracle_encoded_size(dtype, n, N, fmt, MODE_FQ, 1, 1, 0, &cap);
    if (st) return st;
    uint8_t *buf = (uint8_t *)malloc(cap);
    void *y = malloc((size_t)(n ? n : 1) * F.size);
    if (!buf || !y) {
        free(buf);
        free(y);
        return ST_INVALID_ARG;
    }
    int rec = -1, ok_prefix = 1;
    for (int i = 0; i < ncand; ++i) {
        uint64_t bytes;
        st = oracle_encode_mt(x, dtype, n, N, fmt, MODE_FQ, 1, 1, cand[i], SEARCH_BISECT, buf,
                              cap, &bytes, threads);
        if (st) break;
        st = oracle_decode_mt(buf, bytes, y, dtype, n, threads);
        if (st) break;
        double s[6];
        st = oracle_metrics_mt(x, y, dtype, n, N, s, threads);
        if (st) break;
        pts[i].code = cand[i];
        pts[i].flags = 0;
        pts[i].bytes = bytes;
        pts[i].sx = s[0]; pts[i].sy = s[1]; pts[i].sxx = s[2];
        pts[i].sxy = s[3]; pts[i].syy = s[4]; pts[i].sdd = s[5];
        pts[i].r = oracle_corr(s[2], s[3], s[4]);
        if (ok_prefix && pts[i].r >= target) rec = i;
        else ok_prefix = 0;
    }
    free(buf);
    free(y);
    if (st) return st;
    *recommended = rec < 0 ? 0 : rec;
    return rec < 0 ? 1 : ST_OK;
}
