/*
 * CPU ORACLE — test infrastructure only.
 *
 * Plain, slow, obviously-correct reference implementations used to check the
 * CUDA path. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this code; the product library never links or calls it, and it
 * shares no source, header or table with the CUDA path.
 *
 * Contents
 *   1. State-vector update, complex128 (paper Sec. 2.1: a gate on qubits q
 *      multiplies the 2^nq amplitudes whose indices agree outside q by U).
 *   2. QSZ1 block codec, scalar (the project's own absolute-error-bounded
 *      format, standing in for the closed compressor the paper used in
 *      Sec. 4.3 / Sec. 5.1; the bound eb replaces the paper's relative bound).
 *   2b. QSZR block codec, scalar (point-wise relative error bound, Sec. 4.3
 *      Eq. 1-2 and Algorithm 2: sign bitmap with all-0 / all-1 chunk
 *      elision, log-domain quantisation of |x|).
 *   3. Size-predictor MLP, float64 forward / backward / Adam step.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_E_INVALID -1
#define OR_E_CAPACITY -3
#define OR_E_CORRUPT -4
#define OR_E_RANGE -5

/* ====================================================================== */
/* 1. State-vector update (Sec. 2.1, the 1- and 2-qubit update equations,   */
/*    written for any number of target qubits).                              */
/* ====================================================================== */

/* Insert a zero bit at each (ascending) position of `pos` into `x`. */
static uint64_t insert_zero_bits(uint64_t x, const int *pos_sorted, int npos)
{
    for (int i = 0; i < npos; ++i) {
        int p = pos_sorted[i];
        uint64_t low = x & ((1ULL << p) - 1);
        x = ((x >> p) << (p + 1)) | low;
    }
    return x;
}

/*
 * psi: 2^n amplitudes, interleaved (re, im) doubles.
 * q[0..nq-1]: target qubits, q[0] is the least-significant bit of the
 * matrix index. u: 2^nq x 2^nq row-major complex (re, im) doubles.
 * For every index i with zeros at the target bits, gather a_c = psi[i | bits(c)],
 * set psi[i | bits(r)] = sum_c u[r][c] a_c.
 */
int oracle_apply_matrix(double *psi, int n, int nq, const int *q, const double *u)
{
    if (nq < 1 || nq > 10 || nq > n)
        return OR_E_INVALID;
    int sorted[10];
    for (int i = 0; i < nq; ++i) {
        if (q[i] < 0 || q[i] >= n)
            return OR_E_INVALID;
        sorted[i] = q[i];
    }
    for (int i = 0; i < nq; ++i)
        for (int j = i + 1; j < nq; ++j) {
            if (sorted[j] == sorted[i])
                return OR_E_INVALID;
            if (sorted[j] < sorted[i]) {
                int t = sorted[i]; sorted[i] = sorted[j]; sorted[j] = t;
            }
        }
    const int64_t dim = 1LL << nq;
    const int64_t ngroups = 1LL << (n - nq);
    uint64_t offs[1024];
    for (int64_t r = 0; r < dim; ++r) {
        uint64_t o = 0;
        for (int j = 0; j < nq; ++j)
            if ((r >> j) & 1)
                o |= 1ULL << q[j];
        offs[r] = o;
    }
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ngroups; ++g) {
        double ar[1024], ai[1024];
        uint64_t base = insert_zero_bits((uint64_t)g, sorted, nq);
        for (int64_t c = 0; c < dim; ++c) {
            ar[c] = psi[2 * (base | offs[c])];
            ai[c] = psi[2 * (base | offs[c]) + 1];
        }
        for (int64_t r = 0; r < dim; ++r) {
            double sr = 0.0, si = 0.0;
            const double *row = u + 2 * r * dim;
            for (int64_t c = 0; c < dim; ++c) {
                double ur = row[2 * c], ui = row[2 * c + 1];
                sr += ur * ar[c] - ui * ai[c];
                si += ur * ai[c] + ui * ar[c];
            }
            psi[2 * (base | offs[r])] = sr;
            psi[2 * (base | offs[r]) + 1] = si;
        }
    }
    return OR_OK;
}

/* Multiply amplitude |basis> by -1 (Grover oracle / reflection). */
int oracle_apply_phaseflip(double *psi, int n, uint64_t basis)
{
    if (n < 1 || n > 40 || (n < 64 && (basis >> n) != 0))
        return OR_E_INVALID;
    psi[2 * basis] = -psi[2 * basis];
    psi[2 * basis + 1] = -psi[2 * basis + 1];
    return OR_OK;
}

/* |basis> into psi (2^n amplitudes). */
void oracle_init_basis(double *psi, int n, uint64_t basis)
{
    int64_t N = 1LL << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 2 * N; ++i)
        psi[i] = 0.0;
    psi[2 * basis] = 1.0;
}

/* sum |psi_i|^2 */
double oracle_norm_sq(const double *psi, int n)
{
    int64_t N = 1LL << n;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < N; ++i)
        s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

/* <a|b> = sum conj(a_i) b_i, a and b complex128 interleaved (a) and complex64
 * interleaved (b, float). */
void oracle_inner_mixed(const double *a, const float *b, int64_t count, double *re, double *im)
{
    double sr = 0.0, si = 0.0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        double ar = a[2 * i], ai = a[2 * i + 1];
        double br = b[2 * i], bi = b[2 * i + 1];
        sr += ar * br + ai * bi;
        si += ar * bi - ai * br;
    }
    *re = sr;
    *im = si;
}

/* ====================================================================== */
/* 2. QSZ1 codec (scalar).                                                   */
/*                                                                           */
/* Block of N = 2^m complex64 amplitudes, interleaved (re, im).              */
/* Step s = 2^e, e = the largest integer with 2^e <= 2*eb, so s/2 <= eb.     */
/* Code q = round-half-even(x / s); reconstruction x' = q * s, hence         */
/* |x - x'| <= s/2 <= eb for every component (the point-wise bound).         */
/*                                                                           */
/* Stream (little-endian):                                                   */
/*   header 32 B: u32 magic 0x315A5351 ("QSZ1"), u16 version 1, u16 flags 0, */
/*                u8 m, u8 frame_log, i8 e, u8 0, u32 nframes,               */
/*                u64 total_bytes, u64 0                                     */
/*   u32 offsets[nframes + 1] (byte offset of each frame from the stream     */
/*       start; the last entry equals total_bytes), zero-padded to 16 B      */
/*   frames, in order. Frame f holds amplitudes [f*F, (f+1)*F), F =          */
/*   min(4096, N), as C = F/32 chunks of 32 values per plane (plane 0 = Re,  */
/*   plane 1 = Im). Per chunk: d_0 = q_0, d_j = q_j - q_{j-1} (Lorenzo       */
/*   predictor inside the chunk), z = zigzag(d), w = bit length of OR z.     */
/*   A frame whose 2C widths are all zero has length 0. Otherwise:           */
/*   u8 widths[2C] (index plane*C + chunk), zero-padded to 16 B; then for    */
/*   plane 0, 1 and chunk 0..C-1: w words W_b = sum_j bit_b(z_j) << j         */
/*   (b = 0..w-1), u32 each; then zero pad to 16 B.                          */
/* ====================================================================== */

#define QSZ_MAGIC 0x315A5351u
#define QSZ_VERSION 1u
#define QSZ_HEADER 32u
#define QSZ_MAX_FRAME_LOG 12
#define QSZ_MIN_M 5
#define QSZ_MAX_M 26
#define QSZ_E_MIN (-126)
#define QSZ_E_MAX 96

static uint64_t pad16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

static void put_u16(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t *p, uint32_t v)
{
    for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static void put_u64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t get_u16(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
static uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

/* Largest e with 2^e <= 2*eb, found with frexp (no rounding involved):
 * 2*eb = f * 2^x, f in [0.5, 1)  =>  floor(log2(2*eb)) = x - 1. */
int oracle_qsz_step_exponent(double eb, int *e_out)
{
    if (!(eb > 0.0) || !isfinite(eb))
        return OR_E_INVALID;
    int x;
    double f = frexp(2.0 * eb, &x);
    (void)f;
    int e = x - 1;
    if (e < QSZ_E_MIN || e > QSZ_E_MAX)
        return OR_E_INVALID;
    *e_out = e;
    return OR_OK;
}

static int frame_log_for(int m) { return m < QSZ_MAX_FRAME_LOG ? m : QSZ_MAX_FRAME_LOG; }

uint64_t oracle_qsz_worst_case_bytes(int m)
{
    int fl = frame_log_for(m);
    uint64_t F = 1ULL << fl, nframes = 1ULL << (m - fl), C = F / 32;
    return QSZ_HEADER + pad16(4 * (nframes + 1)) + nframes * (pad16(2 * C) + 8 * F);
}

/* Quantise `count` float components with step 2^e. Returns OR_E_INVALID for a
 * non-finite value and OR_E_RANGE if |q| >= 2^30. */
int oracle_qsz_quantize(const float *x, int64_t count, int e, int32_t *q)
{
    double inv_step = ldexp(1.0, -e);
    for (int64_t i = 0; i < count; ++i) {
        if (!isfinite(x[i]))
            return OR_E_INVALID;
        double t = (double)x[i] * inv_step; /* exact: power-of-two scaling */
        double r = nearbyint(t);            /* ties to even (default mode) */
        if (fabs(r) >= 1073741824.0)
            return OR_E_RANGE;
        q[i] = (int32_t)r;
    }
    return OR_OK;
}

static uint32_t zigzag(int32_t d)
{
    uint32_t ud = (uint32_t)d;
    return (ud << 1) ^ (d < 0 ? 0xFFFFFFFFu : 0u);
}

static int32_t unzigzag(uint32_t z)
{
    return (int32_t)((z >> 1) ^ (0u - (z & 1u)));
}

static int bit_length(uint32_t v)
{
    int w = 0;
    while (v) { ++w; v >>= 1; }
    return w;
}

/*
 * Encode one block. amps: 2^m interleaved complex64. On success writes the
 * stream to out (cap bytes) and its length to *out_bytes. If cap is too small
 * returns OR_E_CAPACITY with *out_bytes = the size needed.
 */
int oracle_qsz_encode(const float *amps, int m, double eb, uint8_t *out, uint64_t cap,
                      uint64_t *out_bytes)
{
    if (m < QSZ_MIN_M || m > QSZ_MAX_M)
        return OR_E_INVALID;
    int e;
    int rc = oracle_qsz_step_exponent(eb, &e);
    if (rc)
        return rc;
    const int fl = frame_log_for(m);
    const int64_t N = 1LL << m, F = 1LL << fl, C = F / 32, nframes = N / F;

    /* quantise each plane */
    int32_t *qre = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *qim = (int32_t *)malloc(sizeof(int32_t) * N);
    float *tmp = (float *)malloc(sizeof(float) * N);
    if (!qre || !qim || !tmp) {
        free(qre); free(qim); free(tmp);
        return OR_E_INVALID;
    }
    for (int64_t i = 0; i < N; ++i) tmp[i] = amps[2 * i];
    rc = oracle_qsz_quantize(tmp, N, e, qre);
    if (!rc) {
        for (int64_t i = 0; i < N; ++i) tmp[i] = amps[2 * i + 1];
        rc = oracle_qsz_quantize(tmp, N, e, qim);
    }
    free(tmp);
    if (rc) {
        free(qre); free(qim);
        return rc;
    }

    /* widths and zigzag codes */
    uint32_t *z = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint8_t *w = (uint8_t *)malloc((size_t)(2 * N / 32));
    for (int plane = 0; plane < 2; ++plane) {
        const int32_t *qp = plane ? qim : qre;
        for (int64_t ch = 0; ch < N / 32; ++ch) {
            uint32_t acc = 0;
            for (int j = 0; j < 32; ++j) {
                int64_t i = ch * 32 + j;
                int32_t d = j == 0 ? qp[i] : (int32_t)((uint32_t)qp[i] - (uint32_t)qp[i - 1]);
                uint32_t zz = zigzag(d);
                z[plane * N + i] = zz;
                acc |= zz;
            }
            w[plane * (N / 32) + ch] = (uint8_t)bit_length(acc);
        }
    }
    free(qre); free(qim);

    /* frame lengths and offsets */
    const uint64_t data_start = QSZ_HEADER + pad16(4 * (uint64_t)(nframes + 1));
    uint64_t *offs = (uint64_t *)malloc(sizeof(uint64_t) * (nframes + 1));
    uint64_t pos = data_start;
    for (int64_t f = 0; f < nframes; ++f) {
        offs[f] = pos;
        uint64_t words = 0;
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c)
                words += w[plane * (N / 32) + f * C + c];
        if (words)
            pos += pad16(2 * C) + pad16(4 * words);
    }
    offs[nframes] = pos;
    const uint64_t total = pos;
    *out_bytes = total;
    if (total > cap) {
        free(z); free(w); free(offs);
        return OR_E_CAPACITY;
    }

    memset(out, 0, total);
    put_u32(out + 0, QSZ_MAGIC);
    put_u16(out + 4, QSZ_VERSION);
    put_u16(out + 6, 0);
    out[8] = (uint8_t)m;
    out[9] = (uint8_t)fl;
    out[10] = (uint8_t)(int8_t)e;
    out[11] = 0;
    put_u32(out + 12, (uint32_t)nframes);
    put_u64(out + 16, total);
    put_u64(out + 24, 0);
    for (int64_t f = 0; f <= nframes; ++f)
        put_u32(out + QSZ_HEADER + 4 * f, (uint32_t)offs[f]);

    for (int64_t f = 0; f < nframes; ++f) {
        if (offs[f + 1] == offs[f])
            continue;
        uint8_t *fp = out + offs[f];
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c)
                fp[plane * C + c] = w[plane * (N / 32) + f * C + c];
        uint8_t *wp = fp + pad16(2 * C);
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                int64_t ch = f * C + c;
                int wc = w[plane * (N / 32) + ch];
                for (int b = 0; b < wc; ++b) {
                    uint32_t word = 0;
                    for (int j = 0; j < 32; ++j)
                        word |= ((z[plane * N + ch * 32 + j] >> b) & 1u) << j;
                    put_u32(wp, word);
                    wp += 4;
                }
            }
    }
    free(z); free(w); free(offs);
    return OR_OK;
}

/* Read the header fields; returns OR_E_CORRUPT on a malformed header. */
int oracle_qsz_stream_info(const uint8_t *in, uint64_t in_bytes, int *m, int *e,
                           uint32_t *nframes, uint64_t *total)
{
    if (in_bytes < QSZ_HEADER)
        return OR_E_CORRUPT;
    if (get_u32(in) != QSZ_MAGIC || get_u16(in + 4) != QSZ_VERSION || get_u16(in + 6) != 0)
        return OR_E_CORRUPT;
    *m = in[8];
    *e = (int8_t)in[10];
    *nframes = get_u32(in + 12);
    *total = get_u64(in + 16);
    return OR_OK;
}

/* Decode one block into amps (2^m interleaved complex64). Validates every
 * field; returns OR_E_CORRUPT for any inconsistency. */
int oracle_qsz_decode(const uint8_t *in, uint64_t in_bytes, int m, float *amps)
{
    if (m < QSZ_MIN_M || m > QSZ_MAX_M)
        return OR_E_INVALID;
    int hm, e;
    uint32_t hn;
    uint64_t total;
    if (oracle_qsz_stream_info(in, in_bytes, &hm, &e, &hn, &total))
        return OR_E_CORRUPT;
    const int fl = frame_log_for(m);
    const int64_t N = 1LL << m, F = 1LL << fl, C = F / 32, nframes = N / F;
    if (hm != m || in[9] != fl || in[11] != 0 || hn != (uint32_t)nframes || get_u64(in + 24) != 0)
        return OR_E_CORRUPT;
    if (e < QSZ_E_MIN || e > QSZ_E_MAX)
        return OR_E_CORRUPT;
    const uint64_t data_start = QSZ_HEADER + pad16(4 * (uint64_t)(nframes + 1));
    if (total > in_bytes || total < data_start)
        return OR_E_CORRUPT;
    if (get_u32(in + QSZ_HEADER) != data_start || get_u32(in + QSZ_HEADER + 4 * nframes) != total)
        return OR_E_CORRUPT;
    const float step = ldexpf(1.0f, e);
    for (int64_t f = 0; f < nframes; ++f) {
        uint64_t a = get_u32(in + QSZ_HEADER + 4 * f), b = get_u32(in + QSZ_HEADER + 4 * (f + 1));
        if (b < a || b > total)
            return OR_E_CORRUPT;
        float *dst = amps + 2 * f * F;
        if (a == b) {
            for (int64_t i = 0; i < 2 * F; ++i) dst[i] = 0.0f;
            continue;
        }
        const uint8_t *fp = in + a;
        if (b - a < pad16(2 * C))
            return OR_E_CORRUPT;
        uint64_t words = 0;
        for (int64_t c = 0; c < 2 * C; ++c) {
            if (fp[c] > 32)
                return OR_E_CORRUPT;
            words += fp[c];
        }
        if (words == 0 || b - a != pad16(2 * C) + pad16(4 * words))
            return OR_E_CORRUPT;
        const uint8_t *wp = fp + pad16(2 * C);
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                int wc = fp[plane * C + c];
                uint32_t zc[32];
                for (int j = 0; j < 32; ++j) zc[j] = 0;
                for (int bb = 0; bb < wc; ++bb) {
                    uint32_t word = get_u32(wp);
                    wp += 4;
                    for (int j = 0; j < 32; ++j)
                        zc[j] |= ((word >> j) & 1u) << bb;
                }
                uint32_t acc = 0;
                for (int j = 0; j < 32; ++j) {
                    acc += (uint32_t)unzigzag(zc[j]);
                    dst[2 * (c * 32 + j) + plane] = (float)(int32_t)acc * step;
                }
            }
    }
    return OR_OK;
}

/* ====================================================================== */
/* 2b. QSZR codec (scalar): point-wise RELATIVE error bound (Sec. 4.3,      */
/*     Eq. 1-2, Algorithm 2).                                                */
/*                                                                           */
/* Algorithm 2 records each value's sign in a bitmap, takes |x|, applies     */
/* log2 and compresses the logs under an absolute bound b_a. Here the log2   */
/* of |x| is read off its FP32 bit pattern U = bits(|x|): for a normal       */
/* x = 2^E (1 + M 2^-23), U = (E + 127) 2^23 + M, i.e. 2^23 (E + M 2^-23)    */
/* plus a constant, where E + M 2^-23 is log2|x| with the fraction taken     */
/* linearly (Mitchell's approximation). Its slope d|x| / dL = 2^E <= |x|,    */
/* so an absolute error delta on L moves |x| by at most delta |x| (and by at */
/* most delta / (1 - delta/2) across a binade edge). Quantising U with step  */
/* 2^k, k the largest integer with 2^(k-24) <= b_r / (1 + b_r), therefore    */
/* bounds every normal value's relative error by b_r; Eq. 2's              */
/* b_a = log2(1 + b_r) is the same statement for the exact log2. Integer     */
/* codes keep encoder and decoder exact without a transcendental function.   */
/* Subnormal values (|x| < 2^-126) get an absolute error <= 2^(k-150).       */
/*                                                                           */
/* Per component x: U = bits(|x|); q = (U + 2^(k-1)) >> k; sign s = 1 iff    */
/* x < 0 and q != 0 (Algorithm 2's bitmap: 1 marks a negative value; a value */
/* that reconstructs to zero keeps sign 0); reconstruction |x'| = float with */
/* bits q << k, x' = s ? -|x'| : |x'|. Non-finite x: invalid; |x| >= 2^64:   */
/* out of range.                                                             */
/*                                                                           */
/* Stream: header 32 B as QSZ1 but magic 0x525A5351 ("QSZR") and byte 10 =  */
/* k; offsets[nframes + 1] padded to 16 B; frames of F = min(4096, 2^m)     */
/* amplitudes, C = F/32 chunks per plane, chunk index t = plane*C + chunk.   */
/* Codes q run through the QSZ1 chunk pipeline (Lorenzo delta, zigzag, width,*/
/* bit planes). A frame whose codes are all zero has length 0. Otherwise:    */
/*   u8 widths[2C], padded to 16 B;                                          */
/*   sign chunk types, 2 bits per chunk t (byte t/4, bits 2(t%4)): 0 = all   */
/*     32 signs 0, 1 = all 32 signs 1 (the pre-scan of the sign bitmap       */
/*     that drops all-0 and all-1 chunks), 2 = stored word, 3 = run-coded,   */
/*     padded to 16 B;                                                       */
/*   the sign section, padded to 16 B as a whole: the sign word (bit j =     */
/*     sign of value j) of every type-2 chunk, u32 each, in t order; then    */
/*     one u16 run record per type-3 chunk, in t order;                      */
/*   the code bit planes as in QSZ1, padded to 16 B.                         */
/*                                                                           */
/* Lossless coding of the remaining bitmap (Algorithm 2's last step): a      */
/* chunk whose 32 signs change between neighbours 1 to 3 times (one to three */
/* run boundaries; the transition word T = (W ^ (W >> 1)) & 0x7FFFFFFF has   */
/* 1 to 3 bits set) is type 3 and stores 2 bytes instead of 4: bit 15 = the  */
/* sign of value 0, bits 0-4, 5-9, 10-14 = the boundaries p1 < p2 < p3 in    */
/* 1..31 (value p differs from value p - 1; bit p - 1 of T), unused fields   */
/* zero. Decoding: W = bit 15 ? all ones : 0, then W ^= ~0 << p for every    */
/* nonzero field. A chunk with 4 or more boundaries keeps its raw word.      */
/* ====================================================================== */

#define QSZR_MAGIC 0x525A5351u
#define QSZR_K_MIN 1
#define QSZR_K_MAX 22

/* Largest k with 2^(k-24) <= b_r / (1 + b_r), in [QSZR_K_MIN, QSZR_K_MAX]. */
int oracle_qszr_shift(double rel, int *k_out)
{
    if (!(rel > 0.0) || !(rel < 1.0))
        return OR_E_INVALID;
    const double t = ldexp(rel / (1.0 + rel), 24);
    int x;
    (void)frexp(t, &x); /* t = f 2^x, f in [0.5, 1): floor(log2 t) = x - 1 */
    int k = x - 1;
    while (k > QSZR_K_MIN - 1 && ldexp(1.0, k - 24) > rel / (1.0 + rel)) --k; /* guard the rounding of t */
    if (k < QSZR_K_MIN || k > QSZR_K_MAX)
        return OR_E_INVALID;
    *k_out = k;
    return OR_OK;
}

uint64_t oracle_qszr_worst_case_bytes(int m)
{
    int fl = frame_log_for(m);
    uint64_t F = 1ULL << fl, nframes = 1ULL << (m - fl), C = F / 32;
    return QSZ_HEADER + pad16(4 * (nframes + 1)) +
           nframes * (pad16(2 * C) + pad16((2 * C + 3) / 4) + pad16(8 * C) + 8 * F);
}

static uint32_t f32_bits_or(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}
static float bits_f32_or(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* Codes and signs of `count` components with shift k. */
int oracle_qszr_quantize(const float *x, int64_t count, int k, int32_t *q, uint8_t *sign)
{
    for (int64_t i = 0; i < count; ++i) {
        if (!isfinite(x[i]))
            return OR_E_INVALID;
        const uint32_t U = f32_bits_or(x[i]) & 0x7FFFFFFFu;
        if (U >= 0x5F800000u) /* |x| >= 2^64 */
            return OR_E_RANGE;
        const uint32_t c = (U + (1u << (k - 1))) >> k;
        q[i] = (int32_t)c;
        sign[i] = (uint8_t)(x[i] < 0.0f && c != 0);
    }
    return OR_OK;
}

/* Sign chunk type of sign word w: 0 all clear, 1 all set, 3 run-coded (1..3 boundaries), 2 stored. */
static uint32_t qszr_sign_type(uint32_t w)
{
    if (w == 0u)
        return 0u;
    if (w == 0xFFFFFFFFu)
        return 1u;
    const uint32_t t = (w ^ (w >> 1)) & 0x7FFFFFFFu;
    int r = 0;
    for (int j = 0; j < 31; ++j)
        r += (int)((t >> j) & 1u);
    return r <= 3 ? 3u : 2u;
}

/* Run record of a type-3 sign word: bit 15 = bit 0 of w, then the boundaries in ascending order. */
static uint16_t qszr_run_record(uint32_t w)
{
    uint32_t rec = (w & 1u) << 15, field = 0;
    for (int j = 0; j < 31; ++j)
        if ((((w >> j) ^ (w >> (j + 1))) & 1u) != 0u)
            rec |= (uint32_t)(j + 1) << (5 * field++);
    return (uint16_t)rec;
}

/* Sign word of a run record; 0 with *ok = 0 for a record no encoder writes. */
static uint32_t qszr_run_word(uint32_t rec, int *ok)
{
    const uint32_t p[3] = {rec & 31u, (rec >> 5) & 31u, (rec >> 10) & 31u};
    *ok = p[0] != 0u && (p[1] == 0u ? p[2] == 0u : (p[1] > p[0] && (p[2] == 0u || p[2] > p[1])));
    uint32_t w = (rec >> 15) ? 0xFFFFFFFFu : 0u;
    for (int i = 0; i < 3; ++i)
        if (p[i])
            w ^= 0xFFFFFFFFu << p[i];
    return w;
}

int oracle_qszr_encode(const float *amps, int m, double rel, uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    if (m < QSZ_MIN_M || m > QSZ_MAX_M)
        return OR_E_INVALID;
    int k;
    int rc = oracle_qszr_shift(rel, &k);
    if (rc)
        return rc;
    const int fl = frame_log_for(m);
    const int64_t N = 1LL << m, F = 1LL << fl, C = F / 32, nframes = N / F, NC = N / 32;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * 2 * N);  /* plane-major */
    uint8_t *sg = (uint8_t *)malloc((size_t)(2 * N));
    float *tmp = (float *)malloc(sizeof(float) * N);
    uint32_t *z = (uint32_t *)malloc(sizeof(uint32_t) * 2 * N);
    uint8_t *w = (uint8_t *)malloc((size_t)(2 * NC));
    uint32_t *sw = (uint32_t *)malloc(sizeof(uint32_t) * 2 * NC); /* sign word per chunk */
    uint64_t *offs = (uint64_t *)malloc(sizeof(uint64_t) * (nframes + 1));
    if (!q || !sg || !tmp || !z || !w || !sw || !offs) {
        free(q); free(sg); free(tmp); free(z); free(w); free(sw); free(offs);
        return OR_E_INVALID;
    }
    for (int plane = 0; plane < 2 && !rc; ++plane) {
        for (int64_t i = 0; i < N; ++i) tmp[i] = amps[2 * i + plane];
        rc = oracle_qszr_quantize(tmp, N, k, q + plane * N, sg + plane * N);
    }
    free(tmp);
    if (rc) {
        free(q); free(sg); free(z); free(w); free(sw); free(offs);
        return rc;
    }
    for (int plane = 0; plane < 2; ++plane)
        for (int64_t ch = 0; ch < NC; ++ch) {
            uint32_t acc = 0, s = 0;
            for (int j = 0; j < 32; ++j) {
                const int64_t i = plane * N + ch * 32 + j;
                const int32_t d = j == 0 ? q[i] : (int32_t)((uint32_t)q[i] - (uint32_t)q[i - 1]);
                z[i] = zigzag(d);
                acc |= z[i];
                s |= (uint32_t)sg[i] << j;
            }
            w[plane * NC + ch] = (uint8_t)bit_length(acc);
            sw[plane * NC + ch] = s;
        }
    free(q); free(sg);
    const uint64_t data_start = QSZ_HEADER + pad16(4 * (uint64_t)(nframes + 1));
    const uint64_t tbytes = (uint64_t)(2 * C + 3) / 4;
    uint64_t pos = data_start;
    for (int64_t f = 0; f < nframes; ++f) {
        offs[f] = pos;
        uint64_t words = 0, mixed = 0, runs = 0;
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                const int64_t t = plane * NC + f * C + c;
                const uint32_t type = qszr_sign_type(sw[t]);
                words += w[t];
                mixed += type == 2u;
                runs += type == 3u;
            }
        if (words)
            pos += pad16(2 * C) + pad16(tbytes) + pad16(4 * mixed + 2 * runs) + pad16(4 * words);
    }
    offs[nframes] = pos;
    *out_bytes = pos;
    if (pos > cap) {
        free(z); free(w); free(sw); free(offs);
        return OR_E_CAPACITY;
    }
    memset(out, 0, pos);
    put_u32(out + 0, QSZR_MAGIC);
    put_u16(out + 4, 1);
    put_u16(out + 6, 0);
    out[8] = (uint8_t)m;
    out[9] = (uint8_t)fl;
    out[10] = (uint8_t)k;
    out[11] = 0;
    put_u32(out + 12, (uint32_t)nframes);
    put_u64(out + 16, pos);
    put_u64(out + 24, 0);
    for (int64_t f = 0; f <= nframes; ++f)
        put_u32(out + QSZ_HEADER + 4 * f, (uint32_t)offs[f]);
    for (int64_t f = 0; f < nframes; ++f) {
        if (offs[f + 1] == offs[f])
            continue;
        uint8_t *fp = out + offs[f];
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c)
                fp[plane * C + c] = w[plane * NC + f * C + c];
        uint8_t *tp = fp + pad16(2 * C);
        uint8_t *mp = tp + pad16(tbytes);
        uint64_t mixed = 0, runs = 0;
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c)
                mixed += qszr_sign_type(sw[plane * NC + f * C + c]) == 2u;
        uint8_t *rp = mp + 4 * mixed; /* the run records follow the stored words */
        mixed = 0;
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                const int64_t t = plane * C + c;
                const uint32_t s = sw[plane * NC + f * C + c];
                const uint32_t type = qszr_sign_type(s);
                tp[t / 4] |= (uint8_t)(type << (2 * (t % 4)));
                if (type == 2)
                    put_u32(mp + 4 * mixed++, s);
                else if (type == 3)
                    put_u16(rp + 2 * runs++, qszr_run_record(s));
            }
        uint8_t *wp = mp + pad16(4 * mixed + 2 * runs);
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                const int64_t ch = f * C + c;
                const int wc = w[plane * NC + ch];
                for (int b = 0; b < wc; ++b) {
                    uint32_t word = 0;
                    for (int j = 0; j < 32; ++j)
                        word |= ((z[plane * N + ch * 32 + j] >> b) & 1u) << j;
                    put_u32(wp, word);
                    wp += 4;
                }
            }
    }
    free(z); free(w); free(sw); free(offs);
    return OR_OK;
}

int oracle_qszr_decode(const uint8_t *in, uint64_t in_bytes, int m, float *amps)
{
    if (m < QSZ_MIN_M || m > QSZ_MAX_M)
        return OR_E_INVALID;
    if (in_bytes < QSZ_HEADER || get_u32(in) != QSZR_MAGIC || get_u16(in + 4) != 1 || get_u16(in + 6) != 0)
        return OR_E_CORRUPT;
    const int fl = frame_log_for(m);
    const int64_t N = 1LL << m, F = 1LL << fl, C = F / 32, nframes = N / F;
    const int k = in[10];
    const uint64_t total = get_u64(in + 16);
    if (in[8] != m || in[9] != fl || in[11] != 0 || get_u32(in + 12) != (uint32_t)nframes ||
        get_u64(in + 24) != 0 || k < QSZR_K_MIN || k > QSZR_K_MAX)
        return OR_E_CORRUPT;
    const uint64_t data_start = QSZ_HEADER + pad16(4 * (uint64_t)(nframes + 1));
    if (total > in_bytes || total < data_start)
        return OR_E_CORRUPT;
    if (get_u32(in + QSZ_HEADER) != data_start || get_u32(in + QSZ_HEADER + 4 * nframes) != total)
        return OR_E_CORRUPT;
    const uint64_t tbytes = (uint64_t)(2 * C + 3) / 4;
    for (int64_t f = 0; f < nframes; ++f) {
        const uint64_t a = get_u32(in + QSZ_HEADER + 4 * f), b = get_u32(in + QSZ_HEADER + 4 * (f + 1));
        if (b < a || b > total)
            return OR_E_CORRUPT;
        float *dst = amps + 2 * f * F;
        if (a == b) {
            for (int64_t i = 0; i < 2 * F; ++i) dst[i] = 0.0f;
            continue;
        }
        const uint8_t *fp = in + a;
        if (b - a < pad16(2 * C) + pad16(tbytes))
            return OR_E_CORRUPT;
        uint64_t words = 0, mixed = 0;
        for (int64_t t = 0; t < 2 * C; ++t) {
            if (fp[t] > 32)
                return OR_E_CORRUPT;
            words += fp[t];
        }
        const uint8_t *tp = fp + pad16(2 * C);
        uint64_t runs = 0;
        for (int64_t t = 0; t < 2 * C; ++t) {
            const uint32_t type = (tp[t / 4] >> (2 * (t % 4))) & 3u;
            mixed += type == 2;
            runs += type == 3;
        }
        if (words == 0 || b - a != pad16(2 * C) + pad16(tbytes) + pad16(4 * mixed + 2 * runs) + pad16(4 * words))
            return OR_E_CORRUPT;
        const uint8_t *mp = tp + pad16(tbytes);
        const uint8_t *rp = mp + 4 * mixed;
        const uint8_t *wp = mp + pad16(4 * mixed + 2 * runs);
        for (int plane = 0; plane < 2; ++plane)
            for (int64_t c = 0; c < C; ++c) {
                const int64_t t = plane * C + c;
                const uint32_t type = (tp[t / 4] >> (2 * (t % 4))) & 3u;
                uint32_t s = type == 0 ? 0u : 0xFFFFFFFFu;
                if (type == 2) {
                    s = get_u32(mp);
                    mp += 4;
                } else if (type == 3) {
                    int ok;
                    s = qszr_run_word((uint32_t)rp[0] | ((uint32_t)rp[1] << 8), &ok);
                    rp += 2;
                    if (!ok)
                        return OR_E_CORRUPT;
                }
                const int wc = fp[t];
                uint32_t zc[32];
                for (int j = 0; j < 32; ++j) zc[j] = 0;
                for (int bb = 0; bb < wc; ++bb) {
                    const uint32_t word = get_u32(wp);
                    wp += 4;
                    for (int j = 0; j < 32; ++j) zc[j] |= ((word >> j) & 1u) << bb;
                }
                uint32_t acc = 0;
                for (int j = 0; j < 32; ++j) {
                    acc += (uint32_t)unzigzag(zc[j]);
                    if (acc > (0x5F800000u >> k)) /* no encoder writes a code above 2^64 / 2^k */
                        return OR_E_CORRUPT;
                    const float mag = bits_f32_or(acc << k);
                    dst[2 * (c * 32 + j) + plane] = ((s >> j) & 1u) ? -mag : mag;
                }
            }
    }
    return OR_OK;
}

/* ====================================================================== */
/* 3. Size-predictor MLP, float64.                                           */
/*    y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, x in R^41, hidden 64, 64.   */
/*    Loss = (1/B) sum_b 0.5 (y_b - t_b)^2.                                  */
/*    Flat parameter layout: W1[64][41], b1[64], W2[64][64], b2[64],         */
/*    W3[64], b3[1]  (6913 values).                                          */
/* ====================================================================== */

#define MLP_IN 41
#define MLP_H 64
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

int oracle_mlp_nparams(void) { return MLP_NPARAM; }

void oracle_mlp_forward(const double *p, const double *x, int batch, double *y)
{
    const double *W1 = p, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    for (int s = 0; s < batch; ++s) {
        double h1[MLP_H], h2[MLP_H];
        for (int i = 0; i < MLP_H; ++i) {
            double a = b1[i];
            for (int j = 0; j < MLP_IN; ++j) a += W1[i * MLP_IN + j] * x[s * MLP_IN + j];
            h1[i] = a > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            double a = b2[i];
            for (int j = 0; j < MLP_H; ++j) a += W2[i * MLP_H + j] * h1[j];
            h2[i] = a > 0.0 ? a : 0.0;
        }
        double o = b3[0];
        for (int j = 0; j < MLP_H; ++j) o += W3[j] * h2[j];
        y[s] = o;
    }
}

/* Returns the loss; writes dL/dp into g (same layout as p). */
double oracle_mlp_loss_grad(const double *p, const double *x, const double *t, int batch, double *g)
{
    const double *W1 = p, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
                 *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
    double *gW1 = g, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H,
           *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
    for (int i = 0; i < MLP_NPARAM; ++i) g[i] = 0.0;
    double loss = 0.0;
    for (int s = 0; s < batch; ++s) {
        double a1[MLP_H], h1[MLP_H], a2[MLP_H], h2[MLP_H];
        const double *xs = x + s * MLP_IN;
        for (int i = 0; i < MLP_H; ++i) {
            double a = b1[i];
            for (int j = 0; j < MLP_IN; ++j) a += W1[i * MLP_IN + j] * xs[j];
            a1[i] = a;
            h1[i] = a > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            double a = b2[i];
            for (int j = 0; j < MLP_H; ++j) a += W2[i * MLP_H + j] * h1[j];
            a2[i] = a;
            h2[i] = a > 0.0 ? a : 0.0;
        }
        double o = b3[0];
        for (int j = 0; j < MLP_H; ++j) o += W3[j] * h2[j];
        double r = o - t[s];
        loss += 0.5 * r * r;
        double dy = r / batch;
        gb3[0] += dy;
        double d2[MLP_H], d1[MLP_H];
        for (int j = 0; j < MLP_H; ++j) {
            gW3[j] += dy * h2[j];
            d2[j] = a2[j] > 0.0 ? dy * W3[j] : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            gb2[i] += d2[i];
            for (int j = 0; j < MLP_H; ++j) gW2[i * MLP_H + j] += d2[i] * h1[j];
        }
        for (int j = 0; j < MLP_H; ++j) {
            double a = 0.0;
            for (int i = 0; i < MLP_H; ++i) a += W2[i * MLP_H + j] * d2[i];
            d1[j] = a1[j] > 0.0 ? a : 0.0;
        }
        for (int i = 0; i < MLP_H; ++i) {
            gb1[i] += d1[i];
            for (int j = 0; j < MLP_IN; ++j) gW1[i * MLP_IN + j] += d1[i] * xs[j];
        }
    }
    return loss / batch;
}

/* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). t is 1-based. */
void oracle_adam_step(double *p, const double *g, double *m, double *v, int count, int t,
                      double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
