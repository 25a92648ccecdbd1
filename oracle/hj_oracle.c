/*
 * hj_oracle.c -- plain, single-threaded CPU oracle for the hash-join hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may include, link or call this file.  Only the tests, the
 * smoke check and the bench's CPU-baseline arm use it.  It shares no code with the
 * CUDA path: the hash functions, mixers and layouts below are written here from
 * their published definitions, independently of the kernels.
 *
 * What it computes (He, Lu, He, "Revisiting Co-Processing for Hash Joins on the
 * Coupled CPU-GPU Architecture"):
 *   - the equi-join of R and S (Sec. 3.1, Alg. 1): every pair (r.rid, s.rid) with
 *     r.key == s.key; the output is the matching rid pair (Sec. 5, join selectivity
 *     experiment), so no keys are emitted;
 *   - the radix partitioning of Alg. 2 (Sec. 3.1): tuples split on low bits of the
 *     integer hash value, in one or two passes; the hash is MurmurHash 2.0 (Sec. 5.1).
 *
 * Relations are arrays of <key, rid> tuples (AoS), both fields w bytes wide, w in
 * {4, 8}: two four-byte integer attributes per tuple (Sec. 5.1), widened to eight
 * bytes for the 64-bit workloads.  All arithmetic is unsigned integer arithmetic;
 * sums wrap modulo 2^64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- tuple access */

static uint64_t tup_key(const void *t, int w, uint64_t i)
{
    if (w == 4) return ((const uint32_t *)t)[2 * i];
    return ((const uint64_t *)t)[2 * i];
}

static uint64_t tup_rid(const void *t, int w, uint64_t i)
{
    if (w == 4) return ((const uint32_t *)t)[2 * i + 1];
    return ((const uint64_t *)t)[2 * i + 1];
}

/* ------------------------------------------------------- checksum mixers A, B
 * The join result is summarised by two order-independent sums over the pairs:
 *   c0 = sum A(rid_R) * B(rid_S),  c1 = sum A(rid_R) + B(rid_S)   (mod 2^64).
 * A and B are the 64-bit finaliser of SplitMix64 (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), applied to x and to
 * x XOR a fixed odd constant.  The finaliser is a bijection of 64-bit words. */
static uint64_t sm64_fin(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_mix_a(uint64_t x) { return sm64_fin(x); }
uint64_t oracle_mix_b(uint64_t x) { return sm64_fin(x ^ 0x9E3779B97F4A7C15ULL); }

/* -------------------------------------------------------- MurmurHash 2.0 (Sec. 5.1)
 * Austin Appleby's MurmurHash2, 32-bit variant, over an arbitrary byte string read
 * as little-endian 32-bit blocks: multiply-xorshift-multiply each block into h,
 * fold the tail bytes, then a final avalanche. */
uint32_t oracle_murmur2_32(const void *data, int len, uint32_t seed)
{
    const uint32_t m = 0x5bd1e995u;
    const unsigned char *p = (const unsigned char *)data;
    uint32_t h = seed ^ (uint32_t)len;
    while (len >= 4) {
        uint32_t k = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                     ((uint32_t)p[3] << 24);
        k *= m;
        k ^= k >> 24;
        k *= m;
        h *= m;
        h ^= k;
        p += 4;
        len -= 4;
    }
    if (len > 0) {
        if (len >= 3) h ^= (uint32_t)p[2] << 16;
        if (len >= 2) h ^= (uint32_t)p[1] << 8;
        h ^= (uint32_t)p[0];
        h *= m;
    }
    h ^= h >> 13;
    h *= m;
    h ^= h >> 15;
    return h;
}

/* The 64-bit variant of MurmurHash2 ("MurmurHash64A"): 64-bit blocks, r = 47. */
uint64_t oracle_murmur64a(const void *data, int len, uint64_t seed)
{
    const uint64_t m = 0xc6a4a7935bd1e995ULL;
    const unsigned char *p = (const unsigned char *)data;
    uint64_t h = seed ^ ((uint64_t)len * m);
    int nblocks = len / 8;
    for (int b = 0; b < nblocks; b++) {
        uint64_t k = 0;
        for (int j = 7; j >= 0; j--) k = (k << 8) | p[8 * b + j];
        k *= m;
        k ^= k >> 47;
        k *= m;
        h ^= k;
        h *= m;
    }
    const unsigned char *tail = p + 8 * nblocks;
    int rem = len & 7;
    if (rem > 0) {
        for (int j = rem - 1; j >= 0; j--) h ^= (uint64_t)tail[j] << (8 * j);
        h *= m;
    }
    h ^= h >> 47;
    h *= m;
    h ^= h >> 47;
    return h;
}

/* Hash of one key as the partitioner sees it: the key's w little-endian bytes
 * through MurmurHash2 (w = 4) or MurmurHash64A (w = 8). */
static uint64_t key_hash(uint64_t key, int w, uint64_t seed)
{
    unsigned char b[8];
    for (int j = 0; j < 8; j++) b[j] = (unsigned char)(key >> (8 * j));
    if (w == 4) return oracle_murmur2_32(b, 4, (uint32_t)seed);
    return oracle_murmur64a(b, 8, seed);
}

uint64_t oracle_key_hash(uint64_t key, int w, uint64_t seed) { return key_hash(key, w, seed); }

/* ---------------------------------------------------- equi-join, hash-map form
 * Sec. 3.1, Alg. 1: build a table on R, then look every S tuple up in it and
 * output a rid pair for each build tuple with an equal key.  The table here is a
 * plain chained map (bucket heads + next links), hashed with a Fibonacci
 * multiplier -- deliberately not the kernels' hash; any hash gives the same join.
 * Pairs are written in probe order up to `cap`; the return value is the full
 * number of pairs (so cap = 0 counts only).  Returns -1 on allocation failure. */
int64_t oracle_hash_join(int w, const void *R, uint64_t nR, const void *S, uint64_t nS,
                         uint64_t *out_rid_r, uint64_t *out_rid_s, uint64_t cap)
{
    int bits = 1;
    while (((uint64_t)1 << bits) < 2 * nR) bits++;
    uint64_t nb = (uint64_t)1 << bits;
    int64_t *head = (int64_t *)malloc(nb * sizeof(int64_t));
    int64_t *next = (int64_t *)malloc((nR ? nR : 1) * sizeof(int64_t));
    if (!head || !next) {
        free(head);
        free(next);
        return -1;
    }
    for (uint64_t b = 0; b < nb; b++) head[b] = -1;
    /* build: push each R row onto its bucket's chain */
    for (uint64_t i = 0; i < nR; i++) {
        uint64_t b = (tup_key(R, w, i) * 0x9E3779B97F4A7C15ULL) >> (64 - bits);
        next[i] = head[b];
        head[b] = (int64_t)i;
    }
    /* probe: walk the chain of every S row, compare keys, emit rid pairs */
    uint64_t count = 0;
    for (uint64_t j = 0; j < nS; j++) {
        uint64_t k = tup_key(S, w, j);
        uint64_t b = (k * 0x9E3779B97F4A7C15ULL) >> (64 - bits);
        for (int64_t i = head[b]; i >= 0; i = next[i]) {
            if (tup_key(R, w, (uint64_t)i) == k) {
                if (count < cap) {
                    out_rid_r[count] = tup_rid(R, w, (uint64_t)i);
                    out_rid_s[count] = tup_rid(S, w, j);
                }
                count++;
            }
        }
    }
    free(head);
    free(next);
    return (int64_t)count;
}

/* ---------------------------------------------- equi-join, nested-loop form
 * The definition itself: compare every (r, s) pair.  Only for tiny inputs. */
int64_t oracle_nested_loop_join(int w, const void *R, uint64_t nR, const void *S, uint64_t nS,
                                uint64_t *out_rid_r, uint64_t *out_rid_s, uint64_t cap)
{
    uint64_t count = 0;
    for (uint64_t j = 0; j < nS; j++)
        for (uint64_t i = 0; i < nR; i++)
            if (tup_key(R, w, i) == tup_key(S, w, j)) {
                if (count < cap) {
                    out_rid_r[count] = tup_rid(R, w, i);
                    out_rid_s[count] = tup_rid(S, w, j);
                }
                count++;
            }
    return (int64_t)count;
}

/* --------------------------------------------------------- sort-merge counting
 * Count = sum over keys k of count_R(k) * count_S(k), obtained by sorting both key
 * columns and merging runs of equal keys.  A third, independent route to |J|. */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

int64_t oracle_count_sortmerge(int w, const void *R, uint64_t nR, const void *S, uint64_t nS,
                               uint64_t *count_out)
{
    uint64_t *kr = (uint64_t *)malloc((nR ? nR : 1) * 8);
    uint64_t *ks = (uint64_t *)malloc((nS ? nS : 1) * 8);
    if (!kr || !ks) {
        free(kr);
        free(ks);
        return -1;
    }
    for (uint64_t i = 0; i < nR; i++) kr[i] = tup_key(R, w, i);
    for (uint64_t j = 0; j < nS; j++) ks[j] = tup_key(S, w, j);
    qsort(kr, nR, 8, cmp_u64);
    qsort(ks, nS, 8, cmp_u64);
    uint64_t i = 0, j = 0, count = 0;
    while (i < nR && j < nS) {
        if (kr[i] < ks[j]) {
            i++;
        } else if (kr[i] > ks[j]) {
            j++;
        } else {
            uint64_t k = kr[i], ci = 0, cj = 0;
            while (i < nR && kr[i] == k) i++, ci++;
            while (j < nS && ks[j] == k) j++, cj++;
            count += ci * cj;
        }
    }
    free(kr);
    free(ks);
    *count_out = count;
    return 0;
}

/* ------------------------------------------------------ checksums of the pairs */
void oracle_checksum_pairs(uint64_t n, const uint64_t *rid_r, const uint64_t *rid_s,
                           uint64_t *c_out)
{
    uint64_t c0 = 0, c1 = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t a = oracle_mix_a(rid_r[i]), b = oracle_mix_b(rid_s[i]);
        c0 += a * b;
        c1 += a + b;
    }
    c_out[0] = c0;
    c_out[1] = c1;
}

/* ---------------------------------------------- factorised count and checksums
 * The same three numbers without forming a single pair: group each relation by
 * key (sort on key), keep per key the tuple count and the sum of the mixed rids,
 * and combine matching groups:
 *   count += cR * cS,  c0 += (sum A over R_k) * (sum B over S_k),
 *   c1 += cS * (sum A over R_k) + cR * (sum B over S_k).
 * Used where the pair multiset is too large to materialise. */
typedef struct {
    uint64_t key, mix;
} km_t;

static int cmp_km(const void *a, const void *b)
{
    uint64_t x = ((const km_t *)a)->key, y = ((const km_t *)b)->key;
    return (x > y) - (x < y);
}

int64_t oracle_join_aggregate(int w, const void *R, uint64_t nR, const void *S, uint64_t nS,
                              uint64_t *count_out, uint64_t *c_out)
{
    km_t *r = (km_t *)malloc((nR ? nR : 1) * sizeof(km_t));
    km_t *s = (km_t *)malloc((nS ? nS : 1) * sizeof(km_t));
    if (!r || !s) {
        free(r);
        free(s);
        return -1;
    }
    for (uint64_t i = 0; i < nR; i++) {
        r[i].key = tup_key(R, w, i);
        r[i].mix = oracle_mix_a(tup_rid(R, w, i));
    }
    for (uint64_t j = 0; j < nS; j++) {
        s[j].key = tup_key(S, w, j);
        s[j].mix = oracle_mix_b(tup_rid(S, w, j));
    }
    qsort(r, nR, sizeof(km_t), cmp_km);
    qsort(s, nS, sizeof(km_t), cmp_km);
    uint64_t i = 0, j = 0, count = 0, c0 = 0, c1 = 0;
    while (i < nR && j < nS) {
        if (r[i].key < s[j].key) {
            i++;
        } else if (r[i].key > s[j].key) {
            j++;
        } else {
            uint64_t k = r[i].key, cr = 0, cs = 0, sa = 0, sb = 0;
            while (i < nR && r[i].key == k) sa += r[i].mix, cr++, i++;
            while (j < nS && s[j].key == k) sb += s[j].mix, cs++, j++;
            count += cr * cs;
            c0 += sa * sb;
            c1 += cs * sa + cr * sb;
        }
    }
    free(r);
    free(s);
    *count_out = count;
    c_out[0] = c0;
    c_out[1] = c1;
    return 0;
}

/* ------------------------------------------------------------ radix partition
 * Alg. 2 (Sec. 3.1): every tuple goes to the partition named by low bits of its
 * hash value.  Pass one splits on bits [0, b1); pass two splits each pass-one
 * partition on bits [b1, b1 + b2).  The final partition of a tuple is therefore
 *   p = (h mod 2^b1) * 2^b2 + ((h >> b1) mod 2^b2),
 * and partitions are laid out contiguously in increasing p.  Within a partition
 * tuples keep their input order (a stable counting sort on p).  offsets[p] is the
 * first row of partition p and offsets[2^(b1+b2)] = n. */
int64_t oracle_radix_partition(int w, const void *in, uint64_t n, int b1, int b2, uint64_t seed,
                               void *out, uint64_t *offsets)
{
    if (b1 < 0 || b2 < 0 || b1 + b2 > 24) return -1;
    uint64_t P = (uint64_t)1 << (b1 + b2);
    uint32_t *part = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    uint64_t *cursor = (uint64_t *)calloc(P, sizeof(uint64_t));
    if (!part || !cursor) {
        free(part);
        free(cursor);
        return -1;
    }
    for (uint64_t i = 0; i < n; i++) {
        uint64_t h = key_hash(tup_key(in, w, i), w, seed);
        uint64_t d1 = h & (((uint64_t)1 << b1) - 1);
        uint64_t d2 = (h >> b1) & (((uint64_t)1 << b2) - 1);
        part[i] = (uint32_t)((d1 << b2) | d2);
        cursor[part[i]]++;
    }
    uint64_t run = 0;
    for (uint64_t p = 0; p < P; p++) {
        uint64_t c = cursor[p];
        offsets[p] = run;
        cursor[p] = run;
        run += c;
    }
    offsets[P] = run;
    size_t tb = 2 * (size_t)w;
    for (uint64_t i = 0; i < n; i++) {
        memcpy((char *)out + cursor[part[i]] * tb, (const char *)in + i * tb, tb);
        cursor[part[i]]++;
    }
    free(part);
    free(cursor);
    return 0;
}
