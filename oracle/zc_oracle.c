/*
 * zc_oracle.c -- plain, slow CPU oracle for the error-bounded codec.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library; the two meet only
 * in the byte streams they produce.
 *
 * What it computes (gZCCL, Sec. 3.3.2 adapts an error-bounded GPU compressor;
 * Sec. 3.2.3 and 3.3.3 use it on every ring step).  The paper does not print
 * the compressor's internals; the pipeline below is the prequantize ->
 * blockwise 1-D Lorenzo -> fixed-length bit-plane packing -> prefix-sum
 * placement method, with the readings of every silent point stated where they
 * are used:
 *
 *   q_i   = round(x_i / (2 eb)), exact, ties even prequantization
 *   d_i   = q_i - q_{i-1} inside a block of L,   blockwise Lorenzo delta,
 *           d_{block head} = q_{block head}       head predicted from 0
 *   w_j   = bit length of max_i |d_i| in block j fixed length per block
 *   block j payload: sign plane, then magnitude planes 0 .. w_j-1, each L bits
 *   payload offset of block j = sum of the sizes of blocks before it
 *
 * q is the exactly rounded quotient, so |x - q 2eb| <= eb holds exactly; the
 * reconstruction x^ = fl32(q * 2eb) adds at most half an FP32 ulp of x^.  The
 * file is compiled with -ffp-contract=off so no multiply-add is fused; the
 * relative error bound is resolved in FP64.
 *
 * Stream layout (little-endian):
 *   [0,4)   magic 'Z','C','v','1'
 *   [4]     dtype (0 = f32, 1 = bf16)      [5] log2(L)
 *   [6]     flags (bit 0: raw payload, bit 1: block heads stored apart)
 *   [7]     0
 *   [8,16)  n (u64)   [16,20) eb (f32)   [20,24) nb (u32)
 *   [24,32) payload bytes before padding (u64)
 *   [32, 32+pad16(nb))            width byte per block, zero padded
 *   [.., +pad16(3 nb))            heads-apart streams only: q of every block
 *                                 head, 24-bit two's complement, little-endian
 *   [.., +pad16(P))               block payloads back to back, zero padded
 * where pad16(v) rounds v up to a multiple of 16.
 *
 * Heads apart (flag bit 1; the second format variant): the block head is stored in
 * its fixed 3-byte field and its own delta is taken as 0, so the width covers
 * only d_1 .. d_{L-1}.  Data on a large offset then costs 24 bits per block
 * instead of the offset's bit length on every element.
 *
 * Parity pins live in tests/test_oracle_*.py: hand-derived streams, the closed
 * form of the stream length, exact-rational checks of the quantizer, the
 * elementwise error bound, brute-force round trips on tiny inputs and the
 * special cases (zeros, constants, ramps) whose streams follow by hand.
 * tests/test_oracle_mutants.py plants one mistake at a time in a copy of this
 * file and checks that a pin fails.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_OK 0
#define O_ERR_ARG 1
#define O_ERR_RANGE 2
#define O_ERR_NONFINITE 3
#define O_ERR_CAPACITY 4
#define O_ERR_FORMAT 5

#define O_F32 0
#define O_BF16 1

#define O_HEADER 32u
#define O_MAX_WIDTH 24 /* |q| <= 2^22, so |d| <= 2^23: bit length <= 24 */

static uint64_t pad16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

/* ---- element access ---------------------------------------------------- */

static float bf16_bits_to_float(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* Round-to-nearest-even FP32 -> BF16 (the input to this is always finite). */
static uint16_t float_to_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) /* inf or nan: keep, quiet nan */
        return (uint16_t)((u >> 16) | ((u & 0x007fffffu) ? 0x40u : 0u));
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

static float load_elem(const void* x, uint64_t i, int dtype)
{
    if (dtype == O_F32) return ((const float*)x)[i];
    return bf16_bits_to_float(((const uint16_t*)x)[i]);
}

static void store_elem(void* y, uint64_t i, int dtype, float v)
{
    if (dtype == O_F32) ((float*)y)[i] = v;
    else ((uint16_t*)y)[i] = float_to_bf16_rne(v);
}

static int elem_size(int dtype) { return dtype == O_F32 ? 4 : 2; }

/* ---- error bound -------------------------------------------------------- */

/* The absolute bound as the codec uses it: one FP32 value and its double. */
int zco_qparams(double eb_abs, float* eb, float* two_eb)
{
    if (!(eb_abs > 0.0) || !isfinite(eb_abs)) return O_ERR_ARG;
    float e = (float)eb_abs;
    if (!isnormal(e) || e <= 0.0f) return O_ERR_ARG;
    float t = e + e;
    if (!isfinite(t)) return O_ERR_ARG;
    *eb = e;
    *two_eb = t;
    return O_OK;
}

/* Smallest and largest element; non-finite input is an error. */
int zco_minmax(const void* x, uint64_t n, int dtype, float* mn, float* mx)
{
    float lo = 0.0f, hi = 0.0f;
    for (uint64_t i = 0; i < n; ++i) {
        float v = load_elem(x, i, dtype);
        if (!isfinite(v)) return O_ERR_NONFINITE;
        if (i == 0 || v < lo) lo = v;
        if (i == 0 || v > hi) hi = v;
    }
    *mn = lo;
    *mx = hi;
    return O_OK;
}

/* Relative bound -> absolute, in FP64 from the FP32 extremes (value-range
 * relative bound; a constant input uses max(|max|, 1) as its range). */
double zco_eb_from_rel(double rel, float mn, float mx)
{
    if (mx == mn) {
        double a = fabs((double)mx);
        return rel * (a > 1.0 ? a : 1.0);
    }
    return rel * ((double)mx - (double)mn);
}

/* ---- prequantization ---------------------------------------------------- */

/* q = the integer nearest to x / (2 eb), ties to even, in exact arithmetic.
 * The FP64 quotient of two FP32 values is within 2^-53 (relative) of the
 * exact one while a non-tie quotient below 2^23 is at least 2^-48 (relative)
 * away from the nearest half-integer, so rint() of the FP64 quotient is the
 * exact rounding.  |q| is limited to 2^22, so block deltas fit 24 bits. */
static int quantize_one(float x, float two_eb, int32_t* q_out)
{
    if (!isfinite(x)) return O_ERR_NONFINITE;
    double t = (double)x / (double)two_eb;
    if (!(fabs(t) < 1073741824.0)) return O_ERR_RANGE;
    double r = rint(t);
    if (fabs(r) > 4194304.0) return O_ERR_RANGE;
    *q_out = (int32_t)r;
    return O_OK;
}

int zco_quantize(const void* x, uint64_t n, int dtype, double eb_abs, int32_t* q,
                 uint64_t* bad_index)
{
    float eb, two_eb;
    int st = zco_qparams(eb_abs, &eb, &two_eb);
    if (st) return st;
    for (uint64_t i = 0; i < n; ++i) {
        st = quantize_one(load_elem(x, i, dtype), two_eb, &q[i]);
        if (st) {
            if (bad_index) *bad_index = i;
            return st;
        }
    }
    return O_OK;
}

/* ---- encoding of quantized integers ------------------------------------ */

static void put_u32(uint8_t* p, uint32_t v)
{
    for (int b = 0; b < 4; ++b) p[b] = (uint8_t)(v >> (8 * b));
}
static void put_u64(uint8_t* p, uint64_t v)
{
    for (int b = 0; b < 8; ++b) p[b] = (uint8_t)(v >> (8 * b));
}
static uint32_t get_u32(const uint8_t* p)
{
    uint32_t v = 0;
    for (int b = 0; b < 4; ++b) v |= (uint32_t)p[b] << (8 * b);
    return v;
}
static uint64_t get_u64(const uint8_t* p)
{
    uint64_t v = 0;
    for (int b = 0; b < 8; ++b) v |= (uint64_t)p[b] << (8 * b);
    return v;
}

static int bit_length(uint32_t v)
{
    int w = 0;
    while (v) {
        ++w;
        v >>= 1;
    }
    return w;
}

static void write_header(uint8_t* out, int dtype, int log2L, int flags, uint64_t n, float eb,
                         uint32_t nb, uint64_t payload)
{
    memset(out, 0, O_HEADER);
    out[0] = 'Z';
    out[1] = 'C';
    out[2] = 'v';
    out[3] = '1';
    out[4] = (uint8_t)dtype;
    out[5] = (uint8_t)log2L;
    out[6] = (uint8_t)flags;
    out[7] = 0;
    put_u64(out + 8, n);
    uint32_t ebits;
    memcpy(&ebits, &eb, 4);
    put_u32(out + 16, ebits);
    put_u32(out + 20, nb);
    put_u64(out + 24, payload);
}

/* Delta of element i (0 <= i < L) of block j: the head predicted from 0, or
 * (heads apart) taken as 0; tail padding 0. */
static int32_t block_delta(const int32_t* q, uint64_t n, uint64_t L, uint64_t j, uint64_t i,
                           int heads)
{
    uint64_t e = j * L + i;
    if (e >= n) return 0;
    if (i == 0) return heads ? 0 : q[e];
    return q[e] - q[e - 1];
}

/* Encode the quantized integers q[0..n) into a stream.  eb is only recorded
 * in the header.  Blocks are encoded one after another; the offset of block j
 * is the running (prefix) sum of the sizes of blocks 0..j-1. */
static int encode_q(const int32_t* q, uint64_t n, int dtype, float eb, int log2L, int heads,
                    uint8_t* out, uint64_t cap, uint64_t* out_len)
{
    if (log2L < 4 || log2L > 7 || (dtype != O_F32 && dtype != O_BF16)) return O_ERR_ARG;
    const uint64_t L = 1ull << log2L;
    const uint64_t nb = (n + L - 1) / L;
    if (nb > 0xffffffffull) return O_ERR_ARG;
    const uint64_t wbytes = pad16(nb);
    const uint64_t hbytes = heads ? pad16(3 * nb) : 0;
    const uint64_t payload_at = O_HEADER + wbytes + hbytes;

    /* Pass 1: widths and payload size. */
    uint64_t payload = 0;
    uint8_t* width = (uint8_t*)malloc(nb ? nb : 1);
    if (!width) return O_ERR_ARG;
    for (uint64_t j = 0; j < nb; ++j) {
        uint32_t maxabs = 0;
        for (uint64_t i = 0; i < L; ++i) {
            int32_t di = block_delta(q, n, L, j, i, heads);
            uint32_t a = (uint32_t)(di < 0 ? -(int64_t)di : di);
            if (a > maxabs) maxabs = a;
        }
        int w = bit_length(maxabs);
        if (w > O_MAX_WIDTH) {
            free(width);
            return O_ERR_RANGE;
        }
        width[j] = (uint8_t)w;
        if (w > 0) payload += (uint64_t)(w + 1) * L / 8;
    }
    const uint64_t total = payload_at + pad16(payload);
    *out_len = total;
    if (total > cap) {
        free(width);
        return O_ERR_CAPACITY;
    }
    memset(out, 0, total);
    write_header(out, dtype, log2L, heads ? 2 : 0, n, eb, (uint32_t)nb, payload);
    for (uint64_t j = 0; j < nb; ++j) out[O_HEADER + j] = width[j];
    if (heads) {
        for (uint64_t j = 0; j < nb; ++j) {
            uint32_t h = (uint32_t)q[j * L] & 0xffffffu;  /* |q| <= 2^22: fits 24 bits */
            uint8_t* p = out + O_HEADER + wbytes + 3 * j;
            p[0] = (uint8_t)h;
            p[1] = (uint8_t)(h >> 8);
            p[2] = (uint8_t)(h >> 16);
        }
    }

    /* Pass 2: bit planes. */
    uint64_t off = payload_at;
    const uint64_t plane_bytes = L / 8;
    for (uint64_t j = 0; j < nb; ++j) {
        int w = width[j];
        if (w == 0) continue;
        for (uint64_t i = 0; i < L; ++i) {
            int32_t di = block_delta(q, n, L, j, i, heads);
            uint32_t a = (uint32_t)(di < 0 ? -(int64_t)di : di);
            /* sign plane */
            if (di < 0) out[off + i / 8] |= (uint8_t)(1u << (i % 8));
            /* magnitude planes, least significant first */
            for (int k = 0; k < w; ++k)
                if ((a >> k) & 1u)
                    out[off + (uint64_t)(k + 1) * plane_bytes + i / 8] |= (uint8_t)(1u << (i % 8));
        }
        off += (uint64_t)(w + 1) * plane_bytes;
    }
    free(width);
    return O_OK;
}

int zco_encode_q(const int32_t* q, uint64_t n, int dtype, float eb, int log2L, uint8_t* out,
                 uint64_t cap, uint64_t* out_len)
{
    return encode_q(q, n, dtype, eb, log2L, 0, out, cap, out_len);
}

/* The same with block heads stored apart (stream flag bit 1). */
int zco_encode_q_heads(const int32_t* q, uint64_t n, int dtype, float eb, int log2L,
                       uint8_t* out, uint64_t cap, uint64_t* out_len)
{
    return encode_q(q, n, dtype, eb, log2L, 1, out, cap, out_len);
}

int zco_compress(const void* x, uint64_t n, int dtype, double eb_abs, int log2L, uint8_t* out,
                 uint64_t cap, uint64_t* out_len, uint64_t* bad_index)
{
    float eb, two_eb;
    int st = zco_qparams(eb_abs, &eb, &two_eb);
    if (st) return st;
    if (log2L < 4 || log2L > 7 || (dtype != O_F32 && dtype != O_BF16)) return O_ERR_ARG;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!q) return O_ERR_ARG;
    st = zco_quantize(x, n, dtype, eb_abs, q, bad_index);
    if (!st) st = zco_encode_q(q, n, dtype, eb, log2L, out, cap, out_len);
    free(q);
    return st;
}

int zco_compress_heads(const void* x, uint64_t n, int dtype, double eb_abs, int log2L,
                       uint8_t* out, uint64_t cap, uint64_t* out_len, uint64_t* bad_index)
{
    float eb, two_eb;
    int st = zco_qparams(eb_abs, &eb, &two_eb);
    if (st) return st;
    if (log2L < 4 || log2L > 7 || (dtype != O_F32 && dtype != O_BF16)) return O_ERR_ARG;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!q) return O_ERR_ARG;
    st = zco_quantize(x, n, dtype, eb_abs, q, bad_index);
    if (!st) st = encode_q(q, n, dtype, eb, log2L, 1, out, cap, out_len);
    free(q);
    return st;
}

/* A raw stream: header with the raw flag, then the n elements verbatim. */
int zco_compress_raw(const void* x, uint64_t n, int dtype, uint8_t* out, uint64_t cap,
                     uint64_t* out_len)
{
    if (dtype != O_F32 && dtype != O_BF16) return O_ERR_ARG;
    uint64_t payload = n * (uint64_t)elem_size(dtype);
    uint64_t total = O_HEADER + pad16(payload);
    *out_len = total;
    if (total > cap) return O_ERR_CAPACITY;
    memset(out, 0, total);
    write_header(out, dtype, 5, 1, n, 0.0f, 0u, payload);
    memcpy(out + O_HEADER, x, payload);
    return O_OK;
}

/* ---- decoding ----------------------------------------------------------- */

typedef struct {
    int dtype, log2L, flags;
    uint64_t n, payload;
    uint32_t nb;
    float eb;
} o_header;

static int parse_header(const uint8_t* s, uint64_t len, o_header* h)
{
    if (len < O_HEADER) return O_ERR_FORMAT;
    if (s[0] != 'Z' || s[1] != 'C' || s[2] != 'v' || s[3] != '1') return O_ERR_FORMAT;
    h->dtype = s[4];
    h->log2L = s[5];
    h->flags = s[6];
    if (s[7] != 0 || (h->flags & ~3) != 0 || h->flags == 3) return O_ERR_FORMAT;
    if (h->dtype != O_F32 && h->dtype != O_BF16) return O_ERR_FORMAT;
    h->n = get_u64(s + 8);
    uint32_t ebits = get_u32(s + 16);
    memcpy(&h->eb, &ebits, 4);
    h->nb = get_u32(s + 20);
    h->payload = get_u64(s + 24);
    if (h->flags & 1) {
        if (h->nb != 0 || h->payload != h->n * (uint64_t)elem_size(h->dtype)) return O_ERR_FORMAT;
        if (O_HEADER + pad16(h->payload) > len) return O_ERR_FORMAT;
        return O_OK;
    }
    if (h->log2L < 4 || h->log2L > 7) return O_ERR_FORMAT;
    uint64_t L = 1ull << h->log2L;
    if ((uint64_t)h->nb != (h->n + L - 1) / L) return O_ERR_FORMAT;
    float e = h->eb;
    if (h->nb > 0 && (!isnormal(e) || e <= 0.0f || !isfinite(e + e))) return O_ERR_FORMAT;
    const uint64_t hbytes = (h->flags & 2) ? pad16(3 * (uint64_t)h->nb) : 0;
    if (O_HEADER + pad16(h->nb) + hbytes + pad16(h->payload) > len) return O_ERR_FORMAT;
    uint64_t sum = 0;
    for (uint64_t j = 0; j < h->nb; ++j) {
        int w = s[O_HEADER + j];
        if (w > O_MAX_WIDTH) return O_ERR_FORMAT;
        if (w > 0) sum += (uint64_t)(w + 1) * L / 8;
    }
    if (sum != h->payload) return O_ERR_FORMAT;
    return O_OK;
}

/* Recover the quantized integers: unpack the planes of each block, then an
 * inclusive prefix sum of the deltas inside the block. */
int zco_decode_q(const uint8_t* s, uint64_t len, int32_t* q, uint64_t n)
{
    o_header h;
    int st = parse_header(s, len, &h);
    if (st) return st;
    if (h.n != n || (h.flags & 1)) return O_ERR_FORMAT;
    const uint64_t L = 1ull << h.log2L;
    const uint64_t plane_bytes = L / 8;
    const int heads = (h.flags & 2) != 0;
    const uint64_t head_at = O_HEADER + pad16(h.nb);
    uint64_t off = head_at + (heads ? pad16(3 * (uint64_t)h.nb) : 0);
    for (uint64_t j = 0; j < h.nb; ++j) {
        int w = s[O_HEADER + j];
        int32_t acc = 0;
        if (heads) {  /* the stored head; its delta in the planes is 0 */
            const uint8_t* p = s + head_at + 3 * j;
            uint32_t v = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
            acc = (int32_t)v - ((v & 0x800000u) ? (int32_t)(1 << 24) : 0);  /* 24-bit signed */
        }
        for (uint64_t i = 0; i < L; ++i) {
            int32_t di = 0;
            if (w > 0) {
                uint32_t a = 0;
                for (int k = 0; k < w; ++k)
                    if ((s[off + (uint64_t)(k + 1) * plane_bytes + i / 8] >> (i % 8)) & 1u)
                        a |= 1u << k;
                int neg = (s[off + i / 8] >> (i % 8)) & 1u;
                di = neg ? -(int32_t)a : (int32_t)a;
            }
            acc += di;
            uint64_t e = j * L + i;
            if (e < n) q[e] = acc;
        }
        if (w > 0) off += (uint64_t)(w + 1) * plane_bytes;
    }
    return O_OK;
}

/* Reconstruction x^ = (float)q * 2eb in FP32, stored as f32 or as BF16 (RNE). */
int zco_decompress(const uint8_t* s, uint64_t len, void* out, uint64_t n, int out_dtype)
{
    if (out_dtype != O_F32 && out_dtype != O_BF16) return O_ERR_ARG;
    o_header h;
    int st = parse_header(s, len, &h);
    if (st) return st;
    if (h.n != n) return O_ERR_FORMAT;
    if (h.flags & 1) {
        for (uint64_t i = 0; i < n; ++i)
            store_elem(out, i, out_dtype, load_elem(s + O_HEADER, i, h.dtype));
        return O_OK;
    }
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!q) return O_ERR_ARG;
    st = zco_decode_q(s, len, q, n);
    if (!st) {
        float two_eb = h.eb + h.eb;
        for (uint64_t i = 0; i < n; ++i) store_elem(out, i, out_dtype, (float)q[i] * two_eb);
    }
    free(q);
    return st;
}

/* Stream header fields, for tests: dtype, log2L, flags, n, eb, nb, payload. */
int zco_parse_header(const uint8_t* s, uint64_t len, int* dtype, int* log2L, int* flags,
                     uint64_t* n, float* eb, uint32_t* nb, uint64_t* payload)
{
    o_header h;
    int st = parse_header(s, len, &h);
    if (st) return st;
    *dtype = h.dtype;
    *log2L = h.log2L;
    *flags = h.flags;
    *n = h.n;
    *eb = h.eb;
    *nb = h.nb;
    *payload = h.payload;
    return O_OK;
}

/* ---- one ring reduce-scatter step (Sec. 3.2.3, 3.3.1, 3.3.3) ----------- */

/* Decode the received stream (or take zeros when there is none), add the
 * local chunk in FP32 (decoded + local, one rounding), and re-encode the sum
 * with the fixed absolute bound.  sum_out, when given, receives the FP32 sum;
 * out may be NULL when only the sum is wanted (the last step of the ring). */
int zco_reduce_step(const uint8_t* cin, uint64_t cin_len, const float* local, uint64_t n,
                    double eb_abs, int log2L, uint8_t* out, uint64_t cap, uint64_t* out_len,
                    float* sum_out, uint64_t* bad_index)
{
    float* acc = (float*)malloc(sizeof(float) * (n ? n : 1));
    if (!acc) return O_ERR_ARG;
    int st = O_OK;
    if (cin) {
        st = zco_decompress(cin, cin_len, acc, n, O_F32);
        if (st) {
            free(acc);
            return st;
        }
        for (uint64_t i = 0; i < n; ++i) acc[i] = acc[i] + local[i];
    } else {
        for (uint64_t i = 0; i < n; ++i) acc[i] = local[i];
    }
    if (sum_out) memcpy(sum_out, acc, sizeof(float) * n);
    if (out) st = zco_compress(acc, n, O_F32, eb_abs, log2L, out, cap, out_len, bad_index);
    else {
        for (uint64_t i = 0; i < n; ++i)
            if (!isfinite(acc[i])) {
                st = O_ERR_NONFINITE;
                if (bad_index) *bad_index = i;
                break;
            }
    }
    free(acc);
    return st;
}

/* ---- scatter pack (Sec. 3.3.4, binomial-tree Scatter) ------------------ */

/* Segment p = x[displs[p], displs[p]+counts[p]) is compressed on its own into
 * a complete stream; streams follow each other in p order.  seg_off[p] is
 * where stream p starts, seg_off[P] the total length. */
int zco_scatter_pack(const void* x, int dtype, int P, const uint64_t* counts,
                     const uint64_t* displs, double eb_abs, int log2L, uint8_t* out,
                     uint64_t cap, uint64_t* seg_off)
{
    if (P <= 0) return O_ERR_ARG;
    uint64_t pos = 0;
    int es = elem_size(dtype);
    for (int p = 0; p < P; ++p) {
        seg_off[p] = pos;
        uint64_t len = 0;
        const uint8_t* base = (const uint8_t*)x + displs[p] * (uint64_t)es;
        int st = zco_compress(base, counts[p], dtype, eb_abs, log2L, out + pos,
                              cap > pos ? cap - pos : 0, &len, NULL);
        if (st) return st;
        pos += len;
    }
    seg_off[P] = pos;
    return O_OK;
}
