/*
 * oracle.c -- CPU oracle for the DFR sort path.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may call
 * this file.  It shares no code with the CUDA path and must never be used as
 * a fallback for it.
 *
 * What it computes: the stable ascending order of unsigned integer keys (the
 * payload, 4 or 8 bytes when there is one, travels with its key).  That result has a plain
 * definition, so the oracle writes it out in the most direct radix form the
 * paper describes: a least-significant-digit radix sort built from counting
 * sorts (Preliminaries; Section "Least Significant Digit (LSD) Radix Sorts",
 * Algorithm 1).
 *
 *   - digit width 8 bits, digit j of a key is (key >> 8j) & 255;
 *   - for every digit j = 0, 1, ... (least significant first), one counting
 *     sort: count the digit over the records, turn the counts into starting
 *     indices (exclusive prefix), then deal every record, in input order, to
 *     buf[index[digit]++] (Preliminaries, the count/index/deal description);
 *   - sending area and recipient area swap after every pass; with 4 (u32) or
 *     8 (u64) passes the last deal lands back in the caller's array (Alg. 1,
 *     "final deal back into the original space").
 *
 * Nothing is skipped, diverted or reordered: every pass runs even when its
 * digit is constant, so this file shares no logic with the MSD/diverting path.
 * Stability comes from dealing in input order (LSD stability, Section LSD).
 *
 * Return value: 0 on success, -1 if the scratch buffer cannot be allocated,
 * -2 on a null pointer with n > 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_RADIX_BITS 8
#define ORACLE_BUCKETS 256

/* One counting sort of u32 records on digit j: src -> dst. */
static void counting_pass_u32(const uint32_t* src, uint32_t* dst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    /* count */
    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(src[i] >> shift) & 255u] += 1;
    /* convert the counts into indices: index[d] = sum of count[e], e < d */
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    /* deal, in input order */
    for (i = 0; i < n; ++i) {
        const uint32_t rec = src[i];
        dst[index[(rec >> shift) & 255u]++] = rec;
    }
}

static void counting_pass_u64(const uint64_t* src, uint64_t* dst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(src[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint64_t rec = src[i];
        dst[index[(rec >> shift) & 255u]++] = rec;
    }
}

/* Key-value records: the payload is dealt to the same index as its key. */
static void counting_pass_u64_kv(const uint64_t* ksrc, const uint32_t* vsrc, uint64_t* kdst,
                                 uint32_t* vdst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(ksrc[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint64_t key = ksrc[i];
        const uint64_t at = index[(key >> shift) & 255u]++;
        kdst[at] = key;
        vdst[at] = vsrc[i];
    }
}

static void counting_pass_u32_kv(const uint32_t* ksrc, const uint32_t* vsrc, uint32_t* kdst,
                                 uint32_t* vdst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(ksrc[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint32_t key = ksrc[i];
        const uint64_t at = index[(key >> shift) & 255u]++;
        kdst[at] = key;
        vdst[at] = vsrc[i];
    }
}

/* 64-bit payloads: the same deal, the payload moved as a whole 8-byte word. */
static void counting_pass_u64_kv64(const uint64_t* ksrc, const uint64_t* vsrc, uint64_t* kdst,
                                   uint64_t* vdst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(ksrc[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint64_t key = ksrc[i];
        const uint64_t at = index[(key >> shift) & 255u]++;
        kdst[at] = key;
        vdst[at] = vsrc[i];
    }
}

static void counting_pass_u32_kv64(const uint32_t* ksrc, const uint64_t* vsrc, uint32_t* kdst,
                                   uint64_t* vdst, uint64_t n, int j)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    const int shift = ORACLE_RADIX_BITS * j;

    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(ksrc[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint32_t key = ksrc[i];
        const uint64_t at = index[(key >> shift) & 255u]++;
        kdst[at] = key;
        vdst[at] = vsrc[i];
    }
}

int oracle_sort_u32(uint32_t* keys, uint64_t n)
{
    uint32_t* buf;
    uint32_t* src = keys;
    uint32_t* dst;
    uint32_t* t;
    int j;
    if (n == 0) return 0;
    if (keys == NULL) return -2;
    buf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (buf == NULL) return -1;
    dst = buf;
    for (j = 0; j < 4; ++j) { /* 4 digits: an even count, ends in keys */
        counting_pass_u32(src, dst, n, j);
        t = src; src = dst; dst = t;
    }
    free(buf);
    return 0;
}

int oracle_sort_u64(uint64_t* keys, uint64_t n)
{
    uint64_t* buf;
    uint64_t* src = keys;
    uint64_t* dst;
    uint64_t* t;
    int j;
    if (n == 0) return 0;
    if (keys == NULL) return -2;
    buf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    if (buf == NULL) return -1;
    dst = buf;
    for (j = 0; j < 8; ++j) { /* 8 digits: even, ends in keys */
        counting_pass_u64(src, dst, n, j);
        t = src; src = dst; dst = t;
    }
    free(buf);
    return 0;
}

int oracle_sort_u64_kv(uint64_t* keys, uint32_t* vals, uint64_t n)
{
    uint64_t* kbuf;
    uint32_t* vbuf;
    uint64_t *ks = keys, *kd, *kt;
    uint32_t *vs = vals, *vd, *vt;
    int j;
    if (n == 0) return 0;
    if (keys == NULL || vals == NULL) return -2;
    kbuf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    vbuf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (kbuf == NULL || vbuf == NULL) { free(kbuf); free(vbuf); return -1; }
    kd = kbuf; vd = vbuf;
    for (j = 0; j < 8; ++j) {
        counting_pass_u64_kv(ks, vs, kd, vd, n, j);
        kt = ks; ks = kd; kd = kt;
        vt = vs; vs = vd; vd = vt;
    }
    free(kbuf);
    free(vbuf);
    return 0;
}

int oracle_sort_u32_kv(uint32_t* keys, uint32_t* vals, uint64_t n)
{
    uint32_t* kbuf;
    uint32_t* vbuf;
    uint32_t *ks = keys, *kd, *kt;
    uint32_t *vs = vals, *vd, *vt;
    int j;
    if (n == 0) return 0;
    if (keys == NULL || vals == NULL) return -2;
    kbuf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    vbuf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (kbuf == NULL || vbuf == NULL) { free(kbuf); free(vbuf); return -1; }
    kd = kbuf; vd = vbuf;
    for (j = 0; j < 4; ++j) {
        counting_pass_u32_kv(ks, vs, kd, vd, n, j);
        kt = ks; ks = kd; kd = kt;
        vt = vs; vs = vd; vd = vt;
    }
    free(kbuf);
    free(vbuf);
    return 0;
}

int oracle_sort_u64_kv64(uint64_t* keys, uint64_t* vals, uint64_t n)
{
    uint64_t* kbuf;
    uint64_t* vbuf;
    uint64_t *ks = keys, *kd, *kt;
    uint64_t *vs = vals, *vd, *vt;
    int j;
    if (n == 0) return 0;
    if (keys == NULL || vals == NULL) return -2;
    kbuf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    vbuf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    if (kbuf == NULL || vbuf == NULL) { free(kbuf); free(vbuf); return -1; }
    kd = kbuf; vd = vbuf;
    for (j = 0; j < 8; ++j) {
        counting_pass_u64_kv64(ks, vs, kd, vd, n, j);
        kt = ks; ks = kd; kd = kt;
        vt = vs; vs = vd; vd = vt;
    }
    free(kbuf);
    free(vbuf);
    return 0;
}

int oracle_sort_u32_kv64(uint32_t* keys, uint64_t* vals, uint64_t n)
{
    uint32_t* kbuf;
    uint64_t* vbuf;
    uint32_t *ks = keys, *kd, *kt;
    uint64_t *vs = vals, *vd, *vt;
    int j;
    if (n == 0) return 0;
    if (keys == NULL || vals == NULL) return -2;
    kbuf = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    vbuf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    if (kbuf == NULL || vbuf == NULL) { free(kbuf); free(vbuf); return -1; }
    kd = kbuf; vd = vbuf;
    for (j = 0; j < 4; ++j) {
        counting_pass_u32_kv64(ks, vs, kd, vd, n, j);
        kt = ks; ks = kd; kd = kt;
        vt = vs; vs = vd; vd = vt;
    }
    free(kbuf);
    free(vbuf);
    return 0;
}

/*
 * Key formats: the order a sort by key uses, reduced to the unsigned order of
 * a bijective image of the key's bits (written here from the definitions of
 * two's complement and of IEEE 754 totalOrder, independently of the GPU
 * library).
 *   0 unsigned  the bits as an unsigned integer (identity);
 *   1 signed    two's complement: adding 2^(w-1) modulo 2^w, i.e. flipping
 *               the sign bit, maps [-2^(w-1), 2^(w-1)) monotonically onto
 *               [0, 2^w);
 *   2 float     IEEE 754 binary32 / binary64 totalOrder: a value with the sign
 *               bit clear orders by its magnitude bits, above every value with
 *               the sign bit set, which order by decreasing magnitude bits --
 *               so set the sign bit of a positive value and flip every bit of
 *               a negative one (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN);
 *   flag 0x100  descending: the complement reverses the order of distinct
 *               images; equal keys keep input order (the sort stays stable).
 */
#define ORACLE_FMT_DESC 0x100

static uint64_t fmt_encode(uint64_t x, int bits, int fmt)
{
    const uint64_t all = bits == 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1);
    const uint64_t sign = (uint64_t)1 << (bits - 1);
    const int base = fmt & 0xFF;
    if (base == 1) {
        x = x ^ sign;
    } else if (base == 2) {
        if (x & sign) x = x ^ all;   /* negative: reverse the magnitude order, below every positive */
        else x = x | sign;           /* positive: above every negative */
    }
    if (fmt & ORACLE_FMT_DESC) x = x ^ all;
    return x & all;
}

static uint64_t fmt_decode(uint64_t y, int bits, int fmt)
{
    const uint64_t all = bits == 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1);
    const uint64_t sign = (uint64_t)1 << (bits - 1);
    const int base = fmt & 0xFF;
    if (fmt & ORACLE_FMT_DESC) y = y ^ all;
    if (base == 1) {
        y = y ^ sign;
    } else if (base == 2) {
        if (y & sign) y = y & ~sign; /* was positive */
        else y = y ^ all;            /* was negative */
    }
    return y & all;
}

/* Sort `n` keys of key type `key_type` (0 u32, 1 u64, 2 u64 + u32 payloads,
 * 3 u32 + u32 payloads, 4 u64 + u64 payloads, 5 u32 + u64 payloads) in key
 * format `fmt`: map every key to its image, sort the images with the
 * unsigned LSD sort above, map back.  Returns as the unsigned sorts; -3 for
 * an unknown type or format. */
int oracle_sort_format(int key_type, int fmt, void* keys, void* vals, uint64_t n)
{
    uint64_t i;
    int rc;
    const int base = fmt & 0xFF;
    if ((fmt & ~(0xFF | ORACLE_FMT_DESC)) != 0 || base > 2) return -3;
    if (n == 0) return 0;
    if (keys == NULL) return -2;
    if (key_type == 0 || key_type == 3 || key_type == 5) {
        uint32_t* k = (uint32_t*)keys;
        for (i = 0; i < n; ++i) k[i] = (uint32_t)fmt_encode(k[i], 32, fmt);
        rc = key_type == 0   ? oracle_sort_u32(k, n)
             : key_type == 3 ? oracle_sort_u32_kv(k, (uint32_t*)vals, n)
                             : oracle_sort_u32_kv64(k, (uint64_t*)vals, n);
        for (i = 0; i < n; ++i) k[i] = (uint32_t)fmt_decode(k[i], 32, fmt);
    } else if (key_type == 1 || key_type == 2 || key_type == 4) {
        uint64_t* k = (uint64_t*)keys;
        for (i = 0; i < n; ++i) k[i] = fmt_encode(k[i], 64, fmt);
        rc = key_type == 1   ? oracle_sort_u64(k, n)
             : key_type == 2 ? oracle_sort_u64_kv(k, (uint32_t*)vals, n)
                             : oracle_sort_u64_kv64(k, (uint64_t*)vals, n);
        for (i = 0; i < n; ++i) k[i] = fmt_decode(k[i], 64, fmt);
    } else {
        return -3;
    }
    return rc;
}

/* The single counting sort of the Preliminaries on one digit, exposed so the
 * tests can pin the count/index/deal step by itself (one digit of width 8 at
 * bit position `shift`, u32 records, stable). */
int oracle_counting_pass_u32(const uint32_t* src, uint32_t* dst, uint64_t n, int shift)
{
    uint64_t count[ORACLE_BUCKETS];
    uint64_t index[ORACLE_BUCKETS];
    uint64_t i;
    int d;
    if (n == 0) return 0;
    if (src == NULL || dst == NULL || shift < 0 || shift > 24) return -2;
    for (d = 0; d < ORACLE_BUCKETS; ++d) count[d] = 0;
    for (i = 0; i < n; ++i) count[(src[i] >> shift) & 255u] += 1;
    index[0] = 0;
    for (d = 1; d < ORACLE_BUCKETS; ++d) index[d] = index[d - 1] + count[d - 1];
    for (i = 0; i < n; ++i) {
        const uint32_t rec = src[i];
        dst[index[(rec >> shift) & 255u]++] = rec;
    }
    return 0;
}

/*
 * The estimated deal of Fast Radix (Section "Diverting Fast Radix",
 * Algorithm 3): records are dealt on one 8-bit digit into M = 256 buckets
 * whose sizes are not counted but estimated, each bucket holding `cap`
 * records; a record that finds its bucket full goes to the overflow region
 * instead.  This function plays that deal out record by record, in input
 * order, and returns in *out how many records went to the overflow region.
 * (Keys of `width` 4 or 8 bytes; digit = (key >> shift) & 255.)
 * Returns -2 on a bad argument.
 */
int oracle_overflow_count(const void* keys, uint64_t n, int width, int shift, uint64_t cap, uint64_t* out)
{
    uint64_t fill[ORACLE_BUCKETS];
    uint64_t over = 0;
    uint64_t i;
    int d;
    if (out == NULL || (width != 4 && width != 8) || shift < 0 || shift > 8 * width - 8) return -2;
    if (n > 0 && keys == NULL) return -2;
    for (d = 0; d < ORACLE_BUCKETS; ++d) fill[d] = 0;
    for (i = 0; i < n; ++i) {
        const uint64_t key = width == 4 ? (uint64_t)((const uint32_t*)keys)[i] : ((const uint64_t*)keys)[i];
        const unsigned b = (unsigned)((key >> shift) & 255u);
        if (fill[b] < cap)
            fill[b] += 1; /* lands in its estimated bucket */
        else
            over += 1;    /* the bucket is full: overflow */
    }
    *out = over;
    return 0;
}
