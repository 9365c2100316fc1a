/*
 * Seeded synthetic read generator.
 *
 * This file produces inputs only: upper-case ASCII reads over {A,C,G,T} and
 * nothing else.  It holds none of the SdBG method's arithmetic (no k-mers, no
 * counting, no sorting); both the CUDA path and the CPU oracle consume what it
 * writes.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Every read (or read pair) draws from its own stream, seeded by
 * (seed, stream id), so the output is identical for any thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo_t;

static inline uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

static inline uint64_t xo_next(xo_t *g) {
    uint64_t *s = g->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* One independent stream per (seed, stream). */
static void xo_seed(xo_t *g, uint64_t seed, uint64_t stream) {
    uint64_t x = seed * 0xD1342543DE82EF95ULL + stream;
    uint64_t y = splitmix64_next(&x) ^ stream;
    for (int i = 0; i < 4; i++) g->s[i] = splitmix64_next(&y);
}

static inline double xo_unif(xo_t *g) { return (double)(xo_next(g) >> 11) * 0x1.0p-53; }

/* Uniform integer in [0, n), n >= 1, by rejection (no modulo bias). */
static inline uint64_t xo_below(xo_t *g, uint64_t n) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % n);
    uint64_t r;
    do { r = xo_next(g); } while (r >= lim);
    return r % n;
}

/* Standard normal by the Box-Muller transform. */
static double xo_normal(xo_t *g) {
    double u1 = xo_unif(g), u2 = xo_unif(g);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

/* ---------------------------------------------------------------- genomes */

/* Genome lengths drawn lognormal(log(median), sigma), at least min_len. */
void synth_genome_lengths(uint64_t seed, int n_genomes, double median, double sigma,
                          uint64_t min_len, uint64_t *lens) {
    xo_t g;
    xo_seed(&g, seed, 0x6C656E67ULL);
    for (int i = 0; i < n_genomes; i++) {
        double v = exp(log(median) + sigma * xo_normal(&g));
        uint64_t L = (uint64_t)llround(v);
        lens[i] = L < min_len ? min_len : L;
    }
}

/* Relative abundances drawn lognormal(0, sigma). */
void synth_abundances(uint64_t seed, int n_genomes, double sigma, double *ab) {
    xo_t g;
    xo_seed(&g, seed, 0x61627564ULL);
    for (int i = 0; i < n_genomes; i++) ab[i] = exp(sigma * xo_normal(&g));
}

/* Uniform random bases (codes 0..3, one byte each) for every genome,
 * concatenated in order; genome i uses its own stream. */
void synth_genome_codes(uint64_t seed, int n_genomes, const uint64_t *lens, uint8_t *codes) {
    uint64_t off = 0;
    for (int i = 0; i < n_genomes; i++) {
        xo_t g;
        xo_seed(&g, seed, 0x67656E00ULL + (uint64_t)i);
        uint64_t L = lens[i];
        uint64_t j = 0;
        while (j < L) {
            uint64_t r = xo_next(&g);
            for (int b = 0; b < 32 && j < L; b++, j++) codes[off + j] = (uint8_t)((r >> (2 * b)) & 3);
        }
        off += L;
    }
}

/* ------------------------------------------------------------------ reads */

typedef struct {
    uint64_t seed;
    const uint8_t *genome; /* codes 0..3 */
    int n_genomes;
    const uint64_t *goff; /* n_genomes + 1 offsets into genome */
    const double *cdf;    /* n_genomes cumulative pick weights, last == 1 */
    uint64_t n_units;     /* reads (single-end) or pairs */
    int read_len;
    int paired;
    double insert_mean, insert_sd;
    double err;      /* single-end: iid rate; paired: rate at the 3' end */
    int err_ramp;    /* 1: rate err*(i+0.5)/L at read position i */
    uint8_t *ascii;  /* n_units * (paired ? 2 : 1) * read_len bytes */
    uint64_t begin, end;
} reads_job;

static int pick_genome(xo_t *g, const double *cdf, int n) {
    double u = xo_unif(g);
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (u < cdf[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Write len bases of the genome window [pos, pos+len) to out, reverse
 * complemented when rc != 0, then apply substitutions. */
static void emit_read(xo_t *g, const uint8_t *gen, uint64_t pos, int len, int rc,
                      double err, int ramp, uint8_t *out) {
    for (int i = 0; i < len; i++) {
        uint8_t c = rc ? (uint8_t)(3 - gen[pos + (uint64_t)(len - 1 - i)]) : gen[pos + (uint64_t)i];
        double p = ramp ? err * ((double)i + 0.5) / (double)len : err;
        if (p > 0.0 && xo_unif(g) < p) c = (uint8_t)((c + 1 + xo_below(g, 3)) & 3);
        out[i] = (uint8_t)ACGT[c];
    }
}

static void *reads_worker(void *arg) {
    reads_job *J = (reads_job *)arg;
    const int L = J->read_len;
    for (uint64_t u = J->begin; u < J->end; u++) {
        xo_t g;
        xo_seed(&g, J->seed, 0x7265616400000000ULL + u);
        int gi = pick_genome(&g, J->cdf, J->n_genomes);
        uint64_t gbeg = J->goff[gi], glen = J->goff[gi + 1] - J->goff[gi];
        const uint8_t *gen = J->genome + gbeg;
        if (!J->paired) {
            uint64_t pos = xo_below(&g, glen - (uint64_t)L + 1);
            int rc = (int)(xo_next(&g) >> 63);
            emit_read(&g, gen, pos, L, rc, J->err, J->err_ramp, J->ascii + u * (uint64_t)L);
        } else {
            double ins = J->insert_mean + J->insert_sd * xo_normal(&g);
            uint64_t I = ins < (double)L ? (uint64_t)L : (uint64_t)llround(ins);
            if (I > glen) I = glen;
            uint64_t fpos = xo_below(&g, glen - I + 1);
            int frc = (int)(xo_next(&g) >> 63);
            /* Fragment = genome[fpos, fpos+I) on strand frc.  Mate 1 reads its
             * first L bases; mate 2 reads the reverse complement of its last L. */
            uint8_t *o1 = J->ascii + (2 * u) * (uint64_t)L;
            uint8_t *o2 = o1 + L;
            if (!frc) {
                emit_read(&g, gen, fpos, L, 0, J->err, J->err_ramp, o1);
                emit_read(&g, gen, fpos + I - (uint64_t)L, L, 1, J->err, J->err_ramp, o2);
            } else {
                emit_read(&g, gen, fpos + I - (uint64_t)L, L, 1, J->err, J->err_ramp, o1);
                emit_read(&g, gen, fpos, L, 0, J->err, J->err_ramp, o2);
            }
        }
    }
    return NULL;
}

/* Sample reads from the genomes.  Genome i is picked with probability
 * weight[i] / sum(weight).  Returns 0, or -1 if a genome is shorter than a
 * read. */
int synth_reads(uint64_t seed, const uint8_t *genome, int n_genomes, const uint64_t *lens,
                const double *weight, uint64_t n_units, int read_len, int paired,
                double insert_mean, double insert_sd, double err, int err_ramp,
                uint8_t *ascii, int n_threads) {
    uint64_t *goff = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n_genomes + 1));
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n_genomes);
    double tot = 0.0;
    goff[0] = 0;
    for (int i = 0; i < n_genomes; i++) {
        if (lens[i] < (uint64_t)read_len) { free(goff); free(cdf); return -1; }
        goff[i + 1] = goff[i] + lens[i];
        tot += weight[i];
    }
    double acc = 0.0;
    for (int i = 0; i < n_genomes; i++) { acc += weight[i]; cdf[i] = acc / tot; }
    cdf[n_genomes - 1] = 1.0;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if ((uint64_t)n_threads > n_units) n_threads = n_units ? (int)n_units : 1;
    pthread_t th[256];
    reads_job jobs[256];
    for (int t = 0; t < n_threads; t++) {
        reads_job *J = &jobs[t];
        J->seed = seed; J->genome = genome; J->n_genomes = n_genomes; J->goff = goff; J->cdf = cdf;
        J->n_units = n_units; J->read_len = read_len; J->paired = paired;
        J->insert_mean = insert_mean; J->insert_sd = insert_sd; J->err = err; J->err_ramp = err_ramp;
        J->ascii = ascii;
        J->begin = n_units * (uint64_t)t / (uint64_t)n_threads;
        J->end = n_units * (uint64_t)(t + 1) / (uint64_t)n_threads;
        pthread_create(&th[t], NULL, reads_worker, J);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    free(goff);
    free(cdf);
    return 0;
}
