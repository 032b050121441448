/*
 * Seeded synthetic byte streams for the hashless CDC workloads.
 *
 * This module only draws random numbers and lays out bytes. It holds none
 * of the chunking arithmetic; both the CPU oracle and the GPU path read the
 * buffers it writes.
 *
 * Random source: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used in its counter form,
 * value(key, i) = mix(key + (i + 1) * golden_gamma). Each block of each stream
 * has its own key, so blocks can be generated independently and in parallel
 * with identical results on any host.
 *
 * The paper's datasets (DEB, DEV, LNX, ... in its evaluation section) are not
 * available; these streams stand in for them:
 *   uniform  -- i.i.d. uniform bytes.
 *   mixed    -- 1 MiB blocks, 50% uniform / 30% text-like / 20% zero runs,
 *               in a seeded shuffled order.
 *   edits    -- a version derived from its predecessor by seeded
 *               insert / delete / overwrite runs (dedup-shaped versions).
 *   sizes    -- log-normal file sizes; arrival times -- Poisson process.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_rand(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

/* Key of a sub-stream, derived from (seed, tag, index). */
uint64_t synth_key(uint64_t seed, uint64_t tag, uint64_t index) {
    return mix64(mix64(seed * GAMMA + 0x632BE59BD9B4E019ULL) ^ mix64(tag * 0xD1B54A32D192ED03ULL + index));
}

enum { TAG_UNIFORM = 1, TAG_SHUFFLE = 2, TAG_TEXT = 3, TAG_ZERO = 4, TAG_PERM = 5,
       TAG_RANDBLK = 6, TAG_EDIT = 7, TAG_EDITBYTES = 8, TAG_SIZES = 9, TAG_ARRIVAL = 10,
       TAG_ALG = 11 };

/* ---------- uniform bytes ---------- */

/* Byte i of the uniform stream of `key`: byte (i % 8) of value(key, i / 8). */
static void fill_uniform(uint64_t key, uint64_t offset, uint8_t* out, uint64_t n) {
    uint64_t i = 0;
    while (i < n) {
        uint64_t pos = offset + i;
        uint64_t v = synth_rand(key, pos >> 3);
        unsigned b = (unsigned)(pos & 7);
        for (; b < 8 && i < n; b++, i++) out[i] = (uint8_t)(v >> (8 * b));
    }
}

/* ---------- threading helper ---------- */

typedef void (*range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void* ctx; uint64_t lo, hi; } job_t;
static void* job_run(void* a) { job_t* j = (job_t*)a; j->fn(j->ctx, j->lo, j->hi); return NULL; }

static void parallel_for(uint64_t n, int threads, range_fn fn, void* ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > n) threads = (int)(n ? n : 1);
    pthread_t tid[256];
    job_t jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)threads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    for (int t = 1; t < threads; t++) pthread_create(&tid[t], NULL, job_run, &jobs[t]);
    job_run(&jobs[0]);
    for (int t = 1; t < threads; t++) pthread_join(tid[t], NULL);
}

typedef struct { uint64_t key, offset; uint8_t* out; } uni_ctx;
static void uni_range(void* c, uint64_t lo, uint64_t hi) {
    uni_ctx* u = (uni_ctx*)c;
    fill_uniform(u->key, u->offset + lo, u->out + lo, hi - lo);
}

/* out[k] = byte (offset + k) of the uniform stream of `seed`. */
void synth_uniform(uint64_t seed, uint64_t offset, uint8_t* out, uint64_t n, int threads) {
    uni_ctx c = { synth_key(seed, TAG_UNIFORM, 0), offset, out };
    /* split on 8-byte groups so that threads never share a word */
    if (n < (1u << 20)) { uni_range(&c, 0, n); return; }
    parallel_for(n, threads, uni_range, &c);
}

/* ---------- mixed stream: random / text-like / zero-run blocks ---------- */

/* Zipf(s = 1.1) over 64 ranks: cumulative probabilities scaled to 2^64. */
static const uint64_t ZIPF_CDF[64] = {
0x4020A262F7B6DC00ULL, 0x5E0B43D99AB7DC00ULL, 0x713223A0E1DD9400ULL, 0x7F270448EECB6800ULL,
0x8A123E753B717800ULL, 0x93018400C4EA8000ULL, 0x9A8C0B5EE9454000ULL, 0xA10ED9C9F83B2800ULL,
0xA6C71BA0EB276000ULL, 0xABDF20A67BB78800ULL, 0xB0755AD663137800ULL, 0xB4A067A08EE66800ULL,
0xB8718580C2342000ULL, 0xBBF6251FDDBEB800ULL, 0xBF38F29051E3B000ULL, 0xC2428A47D6E3E800ULL,
0xC519F7F9DD6ED000ULL, 0xC7C5119C1304F000ULL, 0xCA48BA0DFB752000ULL, 0xCCA912CCCE6C8000ULL,
0xCEE9A19CFEBEA800ULL, 0xD10D6D7E02190000ULL, 0xD31715365B6D3000ULL, 0xD508E117C2161000ULL,
0xD6E4D12565CF3000ULL, 0xD8ACA87519781800ULL, 0xDA61F66B493CE000ULL, 0xDC061E4928EC0800ULL,
0xDD9A5D6757C4B000ULL, 0xDF1FD061E5499000ULL, 0xE097776AE087A000ULL, 0xE20239ECD4970000ULL,
0xE360E99DB13C8000ULL, 0xE4B4451BD80DD000ULL, 0xE5FCFA29D0C6B000ULL, 0xE73BA7991D6EB800ULL,
0xE870DEF17EF06000ULL, 0xE99D25DF7EC05800ULL, 0xEAC0F7731A1C8000ULL, 0xEBDCC535D946F000ULL,
0xECF0F81E5A54A800ULL, 0xEDFDF16652890800ULL, 0xEF040B4735A12000ULL, 0xF00399A105C4F800ULL,
0xF0FCEA8E41307800ULL, 0xF1F046E76DEF6000ULL, 0xF2DDF2B863650800ULL, 0xF3C62DA921026800ULL,
0xF4A9335BBE7A7000ULL, 0xF5873BC0C98C7800ULL, 0xF6607B63362FE800ULL, 0xF73523ACDDFCB000ULL,
0xF805632469D49000ULL, 0xF8D165A5640C3000ULL, 0xF999549318CA0000ULL, 0xFA5D5706D5535800ULL,
0xFB1D91FA04FD2800ULL, 0xFBDA286C9AF72800ULL, 0xFC933B882AC81800ULL, 0xFD48EAC005C18800ULL,
0xFDFB53EEA9A7F800ULL, 0xFEAA9370C413F000ULL, 0xFF56C43E06758000ULL, 0xFFFFFFFFFFFFFFFFULL };

#define MIXED_BLOCK (1u << 20)
enum { BLK_RANDOM = 0, BLK_TEXT = 1, BLK_ZERO = 2 };

typedef struct {
    uint64_t seed, nblocks, len;
    uint8_t* types;     /* per block */
    uint8_t perm[64];   /* rank -> byte */
    uint8_t* out;
} mixed_ctx;

static void mixed_block(const mixed_ctx* m, uint64_t b, uint64_t from, uint64_t to, uint8_t* dst) {
    /* writes stream bytes [b*BLOCK + from, b*BLOCK + to) of block b into dst[0..to-from) */
    uint64_t n = to - from;
    switch (m->types[b]) {
    case BLK_RANDOM:
        fill_uniform(synth_key(m->seed, TAG_RANDBLK, b), from, dst, n);
        break;
    case BLK_TEXT: {
        uint64_t key = synth_key(m->seed, TAG_TEXT, b);
        for (uint64_t k = 0; k < n; k++) {
            uint64_t u = synth_rand(key, from + k);
            unsigned r = 0;
            while (r < 63 && u >= ZIPF_CDF[r]) r++;
            dst[k] = m->perm[r];
        }
        break;
    }
    default: { /* zero runs of U[4096, 65536] bytes, each followed by one non-zero byte */
        uint64_t key = synth_key(m->seed, TAG_ZERO, b);
        uint64_t pos = 0, r = 0;
        while (pos < to) {
            uint64_t run = 4096 + synth_rand(key, 2 * r) % (65536 - 4096 + 1);
            uint8_t mark = (uint8_t)(1 + synth_rand(key, 2 * r + 1) % 255);
            uint64_t zlo = pos, zhi = pos + run;            /* zeros */
            for (uint64_t q = (zlo > from ? zlo : from); q < zhi && q < to; q++) dst[q - from] = 0;
            if (zhi >= from && zhi < to) dst[zhi - from] = mark;
            pos = zhi + 1;
            r++;
        }
        break;
    }
    }
}

typedef struct { mixed_ctx* m; uint64_t lo, n; uint8_t* out; } mixed_win;

static void mixed_range(void* c, uint64_t b0, uint64_t b1) {
    /* blocks [b0, b1) of the stream, clipped to the requested window */
    mixed_win* win = (mixed_win*)c;
    for (uint64_t b = b0; b < b1; b++) {
        uint64_t bstart = b * MIXED_BLOCK, bend = bstart + MIXED_BLOCK;
        if (bend > win->m->len) bend = win->m->len;
        uint64_t lo = bstart > win->lo ? bstart : win->lo;
        uint64_t hi = bend < win->lo + win->n ? bend : win->lo + win->n;
        if (lo >= hi) continue;
        mixed_block(win->m, b, lo - bstart, hi - bstart, win->out + (lo - win->lo));
    }
}

static void mixed_setup(mixed_ctx* m, uint64_t seed, uint64_t len) {
    m->seed = seed;
    m->len = len;
    m->nblocks = (len + MIXED_BLOCK - 1) / MIXED_BLOCK;
    m->types = (uint8_t*)malloc(m->nblocks ? m->nblocks : 1);
    uint64_t nb = m->nblocks;
    uint64_t n_rand = (nb + 1) / 2;                 /* 50% */
    uint64_t n_text = (nb * 3 + 5) / 10;            /* 30%, rounded */
    if (n_rand + n_text > nb) n_text = nb - n_rand;
    for (uint64_t b = 0; b < nb; b++)
        m->types[b] = b < n_rand ? BLK_RANDOM : (b < n_rand + n_text ? BLK_TEXT : BLK_ZERO);
    uint64_t key = synth_key(seed, TAG_SHUFFLE, 0);
    for (uint64_t k = nb; k > 1; k--) {            /* Fisher-Yates */
        uint64_t j = synth_rand(key, k) % k;
        uint8_t t = m->types[k - 1]; m->types[k - 1] = m->types[j]; m->types[j] = t;
    }
    for (int r = 0; r < 64; r++) m->perm[r] = (uint8_t)(0x20 + r);
    uint64_t pk = synth_key(seed, TAG_PERM, 0);
    for (int k = 64; k > 1; k--) {
        int j = (int)(synth_rand(pk, (uint64_t)k) % (uint64_t)k);
        uint8_t t = m->perm[k - 1]; m->perm[k - 1] = m->perm[j]; m->perm[j] = t;
    }
}

typedef struct { mixed_win* win; uint64_t b0; } mixed_off;
static void mixed_range_off(void* c, uint64_t lo, uint64_t hi) {
    mixed_off* o = (mixed_off*)c;
    mixed_range(o->win, o->b0 + lo, o->b0 + hi);
}

/* Bytes [lo, lo + n) of the mixed stream whose total length is total_len
 * (1 MiB blocks; the last one may be short; the block order depends on
 * total_len). */
void synth_mixed_range(uint64_t seed, uint64_t total_len, uint64_t lo, uint64_t n,
                       uint8_t* out, int threads) {
    mixed_ctx m;
    memset(&m, 0, sizeof m);
    mixed_setup(&m, seed, total_len);
    mixed_win win = { &m, lo, n, out };
    if (n) {
        uint64_t b0 = lo / MIXED_BLOCK, b1 = (lo + n + MIXED_BLOCK - 1) / MIXED_BLOCK;
        mixed_off oc = { &win, b0 };
        parallel_for(b1 - b0, threads, mixed_range_off, &oc);
    }
    free(m.types);
}

/* The whole mixed stream of `len` bytes. */
void synth_mixed(uint64_t seed, uint8_t* out, uint64_t len, int threads) {
    synth_mixed_range(seed, len, 0, len, out, threads);
}

/* Block type of each 1 MiB block of the mixed stream (0 random, 1 text, 2 zero). */
void synth_mixed_types(uint64_t seed, uint64_t len, uint8_t* types_out) {
    mixed_ctx m;
    memset(&m, 0, sizeof m);
    mixed_setup(&m, seed, len);
    memcpy(types_out, m.types, m.nblocks);
    free(m.types);
}

/* ---------- dedup-shaped versions ---------- */

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}

/* Number of edits so that about frac_ppm parts per million of the bytes are
 * edited (mean run 256.5 bytes). */
uint64_t synth_edit_count(uint64_t len, uint64_t frac_ppm) {
    double edited = (double)len * (double)frac_ppm * 1e-6;
    uint64_t n = (uint64_t)(edited / 256.5 + 0.5);
    return n ? n : 1;
}

/* Upper bound on the output size of synth_edit. */
uint64_t synth_edit_bound(uint64_t len, uint64_t n_edits) { return len + 512 * n_edits; }

/* Apply n_edits seeded edits (uniform over insert / delete / overwrite, run
 * length U[1, 512], positions uniform over the predecessor) to `in`.
 * Returns the new length. */
uint64_t synth_edit(uint64_t seed, const uint8_t* in, uint64_t len, uint64_t n_edits, uint8_t* out) {
    uint64_t key = synth_key(seed, TAG_EDIT, 0);
    uint64_t bkey = synth_key(seed, TAG_EDITBYTES, 0);
    uint64_t* ev = (uint64_t*)malloc(sizeof(uint64_t) * (n_edits ? n_edits : 1));
    for (uint64_t e = 0; e < n_edits; e++) {
        uint64_t pos = len ? synth_rand(key, 3 * e) % len : 0;
        ev[e] = (pos << 16) | (e & 0xFFFF);   /* stable order; edit id in the low bits */
    }
    qsort(ev, n_edits, sizeof(uint64_t), cmp_u64);
    uint64_t cursor = 0, o = 0, nb = 0;
    for (uint64_t k = 0; k < n_edits; k++) {
        uint64_t pos = ev[k] >> 16;
        uint64_t e = k;  /* attributes drawn by sorted rank: deterministic */
        unsigned type = (unsigned)(synth_rand(key, 3 * e + 1) % 3);
        uint64_t run = 1 + synth_rand(key, 3 * e + 2) % 512;
        if (pos < cursor) pos = cursor;
        if (pos > len) pos = len;
        memcpy(out + o, in + cursor, pos - cursor);
        o += pos - cursor;
        cursor = pos;
        if (type == 0) {            /* insert */
            fill_uniform(bkey, nb, out + o, run); nb += run; o += run;
        } else if (type == 1) {     /* delete */
            uint64_t d = run; if (cursor + d > len) d = len - cursor;
            cursor += d;
        } else {                    /* overwrite */
            uint64_t d = run; if (cursor + d > len) d = len - cursor;
            fill_uniform(bkey, nb, out + o, d); nb += d; o += d;
            cursor += d;
        }
    }
    memcpy(out + o, in + cursor, len - cursor);
    o += len - cursor;
    free(ev);
    return o;
}

/* ---------- sizes and arrivals ---------- */

static double unit_open(uint64_t v) { return ((double)(v >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* Log-normal sizes: round(exp(ln(median) + sigma * N(0,1))), clipped to [lo, hi].
 * N(0,1) by the Box-Muller transform. */
void synth_lognormal_sizes(uint64_t seed, uint64_t n, double median, double sigma,
                           uint64_t lo, uint64_t hi, uint64_t* out) {
    uint64_t key = synth_key(seed, TAG_SIZES, 0);
    const double two_pi = 6.283185307179586476925286766559;
    for (uint64_t i = 0; i < n; i++) {
        double u1 = unit_open(synth_rand(key, 2 * i));
        double u2 = unit_open(synth_rand(key, 2 * i + 1));
        double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
        double v = floor(exp(log(median) + sigma * z) + 0.5);
        uint64_t s = v < (double)lo ? lo : (v > (double)hi ? hi : (uint64_t)v);
        out[i] = s;
    }
}

/* Poisson arrivals at `rate` per second: arrival times in seconds. */
void synth_poisson_arrivals(uint64_t seed, uint64_t n, double rate, double* out) {
    uint64_t key = synth_key(seed, TAG_ARRIVAL, 0);
    double t = 0.0;
    for (uint64_t i = 0; i < n; i++) {
        t += -log(unit_open(synth_rand(key, i))) / rate;
        out[i] = t;
    }
}

/* Uniform choice in [0, k) per item. */
void synth_choice(uint64_t seed, uint64_t n, uint32_t k, uint32_t* out) {
    uint64_t key = synth_key(seed, TAG_ALG, 0);
    for (uint64_t i = 0; i < n; i++) out[i] = (uint32_t)(synth_rand(key, i) % k);
}
