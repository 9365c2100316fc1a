/*
 * mh.h - C ABI of the GB300 (sm_103a) SdBG construction library.
 *
 * The library builds the succinct de Bruijn graph (SdBG) of MEGAHIT
 * (Li, Liu, Luo, Sadakane & Lam, "MEGAHIT: an ultra-fast single-node solution
 * for large and complex metagenomics assembly via succinct de Bruijn graph",
 * 2015) from short reads, in four calls that follow the paper's Sec. 2:
 *
 *   mh_pack_reads   reads -> 2-bit codes                (implied by the 2kt-bit
 *                   store of k-mers in Sec. 2, first paragraph)
 *   mh_count_kmers  all (k+1)-mers on both strands, sorted and counted; those
 *                   seen at least d times are solid      (Sec. 2, third para.)
 *   mh_mercy_kmers  mercy (k+1)-mers between a solid edge without outdegree
 *                   and a solid edge without indegree    (Sec. 2, third para.)
 *   mh_build_sdbg   edges sorted in reverse-lexicographic (colex) order of
 *                   their k-prefix, emitted as the BOSS arrays W (minus flag),
 *                   last, F, the validity bit-vector and the zero-indegree
 *                   store                                 (Sec. 2, first and
 *                                                          second paragraphs)
 *
 * All arithmetic is integer and exact.
 *
 * Conventions
 * -----------
 * Symbols: A=0, C=1, G=2, T=3; complement x -> 3-x.  Input bytes may be upper
 * or lower case; any other byte (e.g. N) splits a read into fragments, and no
 * (k+1)-mer crosses a split.
 *
 * Keys: a string s[0..n-1] is the integer sum s[i] * 4^(n-1-i) (first symbol
 * most significant, so integer order is lexicographic order), stored in nw
 * little-endian 64-bit words (word 0 least significant); nw = 1, 2 or 4 for
 * 2(k+1) <= 64, 128 or 256 bits.  Unused high bits are zero.
 *
 * SdBG entry codes in W: $=0, A=1, C=2, G=3, T=4, plus 4 when the minus flag
 * is set (an edge into a target that an earlier entry already enters).
 * Bit-vectors are arrays of uint32 words, entry i at bit (i % 32) of word
 * i / 32; bits past the last entry are zero.
 *
 * Memory and streams
 * ------------------
 * Every call runs on the context's stream, in order.  Outputs are allocated
 * by the library through the context's allocator (the caller's callbacks, or
 * a stream-ordered pool of the context's device) and belong to the returned
 * handle until mh_free_*.  Views return borrowed device pointers, valid while
 * the handle lives.  Calls that must size their output wait once for a small
 * device-to-host copy; all other work is asynchronous.
 *
 * Errors
 * ------
 * Every int-returning call returns MH_OK (0) or a negative MH_E* code; on
 * error no output handle is produced (*out is set to NULL) and the inputs
 * are unchanged.  mh_last_error_message(ctx) describes the last failure.
 * No call aborts the process.  Device-side waits are bounded; a wait that
 * runs out reports MH_ETIMEOUT instead of hanging.
 */
#ifndef MH_H
#define MH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MH_OK 0
#define MH_EINVAL (-1)       /* bad argument: k < 2 or k > 127, d < 1, NULL, k mismatch */
#define MH_ENOMEM (-2)       /* allocation failed or the HBM budget is exceeded */
#define MH_EOVERFLOW (-3)    /* a count or size does not fit its integer type */
#define MH_ETIMEOUT (-4)     /* a bounded device wait ran out */
#define MH_EDEVICE (-5)      /* a CUDA call failed */
#define MH_EUNSUPPORTED (-6) /* the request is valid but not implemented */

typedef struct mh_ctx mh_ctx;
typedef struct mh_reads mh_reads;
typedef struct mh_kmers mh_kmers;
typedef struct mh_sdbg mh_sdbg;
typedef struct mh_contigs mh_contigs;

/* Allocator callbacks.  alloc returns device memory of at least `bytes`
 * bytes, usable in stream order on `stream`, or NULL on failure; free returns
 * it.  `user` is mh_config.alloc_user. */
typedef void* (*mh_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*mh_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct {
    int device;            /* CUDA device ordinal */
    void* stream;          /* cudaStream_t to run on; NULL = a blocking stream the context
                              creates (ordered with the legacy default stream) */
    uint64_t hbm_budget;   /* max bytes the context may hold at once; 0 = no limit */
    mh_alloc_fn alloc;     /* NULL = the library's stream-ordered pool */
    mh_free_fn free;       /* must be set iff alloc is set */
    void* alloc_user;
    int with_mult;         /* 1: mh_build_sdbg also emits mult[] (edge counts) */
    int profile;           /* 1: time every kernel launch with CUDA events */
} mh_config;

/* Create a context on cfg->device.  Returns MH_OK and *out, or an error. */
int mh_create(const mh_config* cfg, mh_ctx** out);
void mh_destroy(mh_ctx* ctx);

/* ---------------------------------------------------------------- reads */

/* Pack reads into 2-bit codes, split at bytes outside ACGTacgt.
 *   ascii      n_bases bytes: all reads back to back (host or device memory)
 *   offs       n_reads + 1 uint64 offsets into ascii, non-decreasing,
 *              offs[0] = 0, offs[n_reads] = n_bases (same memory kind as ascii)
 *   on_device  1 if ascii and offs are device pointers, 0 if host pointers
 *              (host memory is copied in on the context's stream; pinned
 *              memory makes that copy asynchronous)
 * The handle holds the fragments (maximal runs of valid bases, empty reads
 * contribute none) packed back to back: base j of the packed stream at bits
 * 31-2(j%16) of word j/16, frag_offs[f]..frag_offs[f+1] the bases of fragment
 * f, frag_read[f] its read.  Errors: MH_EINVAL (NULL pointer, offs not
 * monotone), MH_ENOMEM. */
int mh_pack_reads(mh_ctx* ctx, const uint8_t* ascii, uint64_t n_bases, const uint64_t* offs,
                  uint64_t n_reads, int on_device, mh_reads** out);

typedef struct {
    uint64_t n_reads, n_bases;  /* as given */
    uint64_t n_frags;           /* fragments */
    uint64_t n_packed;          /* bases in the packed stream (valid bases) */
    const uint32_t* packed;     /* device, ceil(n_packed/16) words (+ zero padding) */
    const uint64_t* frag_offs;  /* device, n_frags + 1 */
    const uint32_t* frag_read;  /* device, n_frags */
} mh_reads_view;
int mh_reads_view_get(const mh_reads* r, mh_reads_view* v);
void mh_free_reads(mh_reads* r);

/* ------------------------------------------------------------ counting */

/* Count every (k+1)-mer of every fragment on both strands (each window adds
 * one to itself and one to its reverse complement, so a palindromic (k+1)-mer
 * gains two) and keep those with count >= d: the solid (k+1)-mers, sorted
 * ascending, closed under reverse complement, with exact uint32 counts.
 * 2 <= k <= 127, d >= 1.  The handle also keeps the sorted count spectrum
 * that mh_mercy_kmers needs.  Errors: MH_EINVAL, MH_ENOMEM, MH_EOVERFLOW (a
 * count above 2^32-1), MH_ETIMEOUT, MH_EDEVICE. */
int mh_count_kmers(mh_ctx* ctx, const mh_reads* reads, int k, int d, mh_kmers** solid_out);

/* Mercy (k+1)-mers.  Degrees are those of the solid graph: x has no
 * outdegree if no solid edge starts with x[1..k]; y has no indegree if no
 * solid edge ends with y[0..k-1].  In each fragment, forward strand, for two
 * consecutive solid positions p < q with q > p+1, x = edge p without
 * outdegree and y = edge q without indegree, the edges at p+1..q-1 are mercy
 * edges.  The result is closed under reverse complement, sorted, disjoint
 * from the solid set, and carries each edge's count from mh_count_kmers (in
 * [1, d-1]).  `solid` must come from mh_count_kmers on the same reads.
 * Errors: MH_EINVAL, MH_ENOMEM, MH_ETIMEOUT, MH_EDEVICE. */
int mh_mercy_kmers(mh_ctx* ctx, const mh_reads* reads, const mh_kmers* solid, mh_kmers** mercy_out);

typedef struct {
    int k, nw;                /* (k+1)-mers, nw words per key */
    uint64_t n;               /* keys */
    const uint64_t* keys;     /* device, n * nw words, ascending */
    const uint32_t* counts;   /* device, n */
    uint64_t n_kmers;         /* |K|: all (k+1)-mers on both strands (counting handles) */
    uint64_t n_distinct;      /* distinct (k+1)-mers in K (counting handles) */
} mh_kmers_view;
int mh_kmers_view_get(const mh_kmers* s, mh_kmers_view* v);
void mh_free_kmers(mh_kmers* s);

/* ---------------------------------------------------------------- SdBG */

/* Build the BOSS arrays of the edge set E = solid + mercy (mercy may be
 * NULL).  Entries are E plus padding, in colex order: node symbols k-1 down
 * to 0, then the label, with $ below every base.
 *   * every zero-indegree node v gets ONE dummy entry: node $ v[0..k-2],
 *     label v[k-1]; v is stored in aux (nw words each, k symbols), in the
 *     order of the dummy entries (t of them, so aux is the 2kt-bit store);
 *   * every node with no outgoing edge gets one entry labelled $ (u of them);
 *   * last[i] = 1 iff entry i is its node's final entry; dummy[i] marks the
 *     dummy entries; valid[i] = 1 for every entry;
 *   * F[c] = number of entries whose node ends with a symbol below c, for c
 *     in $ A C G T, and F[5] = m.
 * Errors: MH_EINVAL (k mismatch), MH_ENOMEM, MH_ETIMEOUT, MH_EDEVICE. */
int mh_build_sdbg(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, mh_sdbg** out);

typedef struct {
    int k, nw;
    uint64_t m;               /* entries */
    uint64_t t;               /* dummy entries = zero-indegree nodes */
    uint64_t u;               /* $ entries = zero-outdegree nodes */
    uint64_t n_nodes;         /* popcount(last) */
    uint64_t F[6];            /* host copy */
    const uint8_t* W;         /* device, m */
    const uint32_t* last;     /* device, ceil(m/32) words */
    const uint32_t* valid;    /* device, ceil(m/32) words */
    const uint32_t* dummy;    /* device, ceil(m/32) words */
    const uint64_t* aux;      /* device, t * nw words */
    const uint32_t* mult;     /* device, m, or NULL unless with_mult */
} mh_sdbg_view;
int mh_sdbg_view_get(const mh_sdbg* g, mh_sdbg_view* v);
void mh_free_sdbg(mh_sdbg* g);

/* The graph in one flat little-endian file ("MHSDBG01", a header with k, nw,
 * m, t, u, the node count and F, then W, last, valid, dummy, aux and mult
 * when present, then an FNV-1a hash of every byte before it), so that it
 * outlives the process.  mh_sdbg_save waits for the graph's stream and
 * copies through host memory.  mh_sdbg_load checks the magic, the header
 * and the sizes against the file's length before it allocates, and the hash
 * after reading; the graph it returns is owned by the caller (mh_free_sdbg)
 * and lives on ctx's device.  Errors: MH_EINVAL (NULL, a file that cannot
 * be opened, written or read, or that is not a whole, undamaged graph file;
 * nothing is returned then), MH_ENOMEM, MH_EDEVICE. */
int mh_sdbg_save(const mh_sdbg* g, const char* path);
int mh_sdbg_load(mh_ctx* ctx, const char* path, mh_sdbg** out);

/* ------------------------------------------- multiple-k iteration */

/* The paper (Sec. 2 fourth paragraph, Sec. 3) builds the graph for a list of
 * increasing k and carries the contigs of each k into the graph of the next.
 * Graph cleaning and contig assembly are outside this library; a contig here
 * is a random walk of the graph E = solid + mercy (mercy may be NULL):
 *   r(w, j)   SplitMix64 output number (w << 24) + j of the stream seeded
 *             with `seed` (state advanced by 0x9E3779B97F4A7C15, output
 *             z ^= z >> 30, z *= 0xBF58476D1CE4E5B9, z ^= z >> 27,
 *             z *= 0x94D049BB133111EB, z ^= z >> 31);
 *   walk w    starts at edge r(w, 0) mod |E| of solid followed by mercy (each
 *             in ascending order), its k+1 symbols; step j = 1, 2, ... takes
 *             the out-edges of the walk's last k symbols (the edges of E with
 *             that k-prefix) in label order, stops if there are none, else
 *             appends the label of out-edge r(w, j) mod (their number); a
 *             walk stops at max_len symbols.
 * Contig w is walk w (n_walks contigs, none if E is empty), as ACGT bytes.
 * k + 1 <= max_len < 2^24, n_walks < 2^40.  Errors: MH_EINVAL, MH_ENOMEM,
 * MH_EDEVICE. */
int mh_walk_contigs(mh_ctx* ctx, const mh_kmers* solid, const mh_kmers* mercy, uint64_t n_walks, uint64_t max_len,
                    uint64_t seed, mh_contigs** out);

typedef struct {
    int k;                    /* the graph's k */
    uint64_t n;               /* contigs */
    uint64_t n_bases;         /* bases of all contigs */
    const uint8_t* ascii;     /* device, n_bases bytes, 'A' 'C' 'G' 'T' */
    const uint64_t* offs;     /* device, n + 1 offsets into ascii */
} mh_contigs_view;
int mh_contigs_view_get(const mh_contigs* c, mh_contigs_view* v);
void mh_free_contigs(mh_contigs* c);

/* mh_pack_reads on device buffers, with `copies` copies of every contig of
 * `contigs` (may be NULL) appended as reads: copy c of contig i is read
 * n_reads + i * copies + c.  With copies = d every (k'+1)-mer of a contig is
 * solid at the next k' (the contig-derived edges).  Errors: as
 * mh_pack_reads. */
int mh_pack_reads_contigs(mh_ctx* ctx, const uint8_t* ascii, uint64_t n_bases, const uint64_t* offs,
                          uint64_t n_reads, const mh_contigs* contigs, int copies, mh_reads** out);

/* ------------------------------------------------------ batched sets */

/* One read set of a batch: reads back to back with n_reads + 1 offsets, as
 * for mh_pack_reads; on_device = 1 when ascii and offs are device pointers
 * (they must stay valid and unchanged until mh_run_batch returns). */
typedef struct {
    const uint8_t* ascii;
    uint64_t n_bases;
    const uint64_t* offs;
    uint64_t n_reads;
    int on_device;
} mh_read_set;

/* The outputs of one set: handles as mh_count_kmers, mh_mercy_kmers and
 * mh_build_sdbg return them (NULL where the flags skip the step or the set
 * failed), owned by the caller (mh_free_*, before mh_destroy of the
 * context), and the set's status (MH_OK or the error of its first failing
 * step; a failed set keeps no outputs). */
typedef struct {
    mh_kmers* solid;
    mh_kmers* mercy;
    mh_sdbg* sdbg;
    int status;
} mh_set_result;

#define MH_BATCH_MERCY 1     /* run mh_mercy_kmers on each set */
#define MH_BATCH_BUILD 2     /* run mh_build_sdbg (solid + mercy) on each set */
#define MH_BATCH_AUTOTUNE 4  /* time counting plans once per context, key width, k and size class */

/* Run the whole path (Sec. 2, paragraphs 1-3: pack, count with the solid
 * filter, mercy, SdBG) on n_sets independent read sets, each an independent
 * problem, k and d shared.  `workers` (1..64) host threads each drive a
 * worker context of ctx (its own stream and stream-ordered pool, created on
 * first use and kept until mh_destroy) and take sets largest first; a set
 * starts when its estimated working set fits ctx's HBM budget (without one,
 * 85% of the device's memory) next to the sets in flight, or when none is.
 * Sets run concurrently on the workers' streams.  Work on ctx's stream before
 * the call is ordered before every set; ctx's stream waits for every set's
 * last kernel, so work queued on it after the call sees all outputs.  With
 * profiling on, the workers' kernel statistics are added to ctx's.
 * MH_BATCH_AUTOTUNE: before the first batch at a given key width, k and size
 * class (log2 of the largest set's bases, halved), counts the largest set
 * once with each of a set of counting plans (mh_count_plan: path, scatter
 * tile shape, unit or spread bits, out-of-core buckets when the set needs
 * them) and keeps the fastest for the context (mh_get_count_plan reports
 * it).  Returns MH_OK when every set
 * succeeded, else the first failing set's error (out[i].status tells which).
 * Not to be called concurrently on one context.  Errors: MH_EINVAL (NULL
 * pointers, n_sets < 0, workers outside 1..64, k or d out of range). */
int mh_run_batch(mh_ctx* ctx, const mh_read_set* sets, int n_sets, int k, int d, int workers, int flags,
                 mh_set_result* out);

/* Peak device bytes the library plans for one read set through the whole
 * path at this k (counting dominates: about 48 bytes per window and key
 * word, plus the packed reads, 512 MB of upload staging for host input and
 * 64 MB); what mh_run_batch and the server admit jobs by.  0 for NULL or k
 * outside 2..127. */
uint64_t mh_job_bytes(const mh_read_set* set, int k);

/* ------------------------------------------------------------ serving */

/* A request server (Sec. 2's whole path per request): jobs (one read set,
 * k, d) are submitted at any time and taken first in, first out by `slots`
 * worker threads, each driving a worker context of its own (its own stream
 * and stream-ordered pool on ctx's device, created with the server).  A job
 * is admitted when a slot is free and its mh_job_bytes estimate fits
 * `hbm_budget` next to the jobs running and the results still held, or
 * when nothing is held (a job larger than the budget runs alone).  A job's
 * result (solid and mercy tables, SdBG, by the MH_BATCH_* flags) stays on
 * the device, counted against the budget, until mh_server_release; with
 * MH_SERVE_AUTO_RELEASE it is freed when the job ends.  MH_SERVE_DRY_RUN
 * runs no device work (ctx may be NULL): a job takes n_reads microseconds
 * on the host and gives no outputs, so the scheduling can be tested without
 * a GPU.  The read set's memory must stay valid until the job has ended. */
typedef struct mh_server mh_server;

/* A job's record.  Times in seconds on the server's steady clock. */
typedef struct {
    double submit_s;
    double start_s;    /* -1 until admitted */
    double end_s;      /* -1 until ended */
    int slot;          /* worker that ran it, -1 until admitted */
    int status;        /* MH_OK, or the error of its first failing step */
    uint64_t est_bytes;
} mh_job_info;

#define MH_SERVE_AUTO_RELEASE 8
#define MH_SERVE_DRY_RUN 16

/* Errors: MH_EINVAL (NULL out, slots outside 1..64, no ctx without
 * MH_SERVE_DRY_RUN), MH_ENOMEM / MH_EDEVICE (a worker context failed). */
int mh_server_create(mh_ctx* ctx, int slots, uint64_t hbm_budget, int flags, mh_server** out);
/* Queues a job; *job gets its id.  MH_EINVAL for NULL arguments, k outside
 * 2..127 or d < 1, or after mh_server_destroy has begun. */
int mh_server_submit(mh_server* s, const mh_read_set* set, int k, int d, uint64_t* job);
/* Waits up to timeout_s seconds (< 0: without limit) for the job to end.
 * MH_OK once it has ended: out (if not NULL) gets its handles, owned by the
 * server (NULL when released, failed or skipped), info (if not NULL) its
 * record, whose status is the job's own result.  MH_ETIMEOUT if it has not
 * ended in time; MH_EINVAL for an unknown or released id. */
int mh_server_wait(mh_server* s, uint64_t job, double timeout_s, mh_set_result* out, mh_job_info* info);
/* Frees an ended job's result, returns its bytes to the budget and drops
 * its record.  MH_EINVAL for an unknown id or a job still queued or running. */
int mh_server_release(mh_server* s, uint64_t job);
/* Bytes held now (running jobs and unreleased results, by estimate), the
 * most ever held, jobs queued and running.  Any pointer may be NULL. */
int mh_server_stats(mh_server* s, uint64_t* held_bytes, uint64_t* max_held_bytes, uint64_t* queued,
                    uint64_t* running);
/* Starts the most-held figure of mh_server_stats again from what is held
 * now (to measure one stream of jobs on a server kept warm). */
int mh_server_reset_max(mh_server* s);
/* Worker context `slot` (its kernel statistics, mh_trim); NULL for a dry
 * run or a slot out of range.  Owned by the server. */
mh_ctx* mh_server_context(mh_server* s, int slot);
/* Lets every queued and running job end (the results of ended jobs are
 * freed first, so that queued jobs find room), frees all results, the
 * worker contexts and the server. */
int mh_server_destroy(mh_server* s);

/* The scatter-pass tile shape the context uses for 1-word keys: 0 = 16 keys
 * a thread at 3 CTAs per SM (the default), 1 = 12 at 4, 2 = 14 at 3; -1
 * before any autotuning (the default applies). */
int mh_sort_shape(const mh_ctx* ctx);

/* How the context counts (Sec. 2, third paragraph: the sort and count of
 * every (k+1)-mer).  Every plan gives the same results; only the route and
 * its speed change.  -1 / 0 fields mean the library's default.
 *   path              0: unit counting (8-bit passes over the top bits of
 *                     the mixed keys, then each unit of about 160 / 96 / 56
 *                     keys (1 / 2 / 4 key words) sorted and counted by one
 *                     warp); 1: the spread sort (passes over the top
 *                     ceil(log2 n) bits, a fix-up of keys sharing them, a run
 *                     pass)
 *   sort_shape        the scatter tile shape (see mh_sort_shape)
 *   unit_bits_delta   added to the unit bits of path 0 (-2..2)
 *   spread_bits_delta added to the bits path 1 sorts by passes (-8, 0, 8)
 *   bucket_bits       out-of-core buckets: 2^bucket_bits (0..6), -1 = the
 *                     memory plan's choice
 * MH_BATCH_AUTOTUNE tries a set of plans on the largest set of a batch (per
 * key width, k and size class of that set) and keeps the fastest.
 * Errors: MH_EINVAL (NULL, a field out of range). */
typedef struct {
    int path;
    int sort_shape;
    int unit_bits_delta;
    int spread_bits_delta;
    int bucket_bits;
} mh_count_plan;
int mh_get_count_plan(const mh_ctx* ctx, mh_count_plan* out);
int mh_set_count_plan(mh_ctx* ctx, const mh_count_plan* plan);

/* ------------------------------------------------- no-allocation sort */

/* Sort n keys (nw = 1, 2 or 4 words each, layout as above) ascending by their
 * low key_bits bits (1 <= key_bits <= 64 * nw; higher bits must be zero),
 * reading keys_in and writing keys_out (distinct device buffers of n * nw
 * words on the calling thread's current device, 8-byte aligned for nw = 1 and
 * 16-byte aligned for nw = 2 or 4), on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The paper has no
 * counterpart: this is the library's radix sort, offered to callers that may
 * not allocate device memory at all - hosts that own the device's whole
 * memory budget, or code that must never enter the driver's allocator or
 * synchronise the device the way cudaFree does.  It calls no cudaMalloc,
 * cudaFree or other allocating routine; all scratch space is one static
 * device array of about 17 MiB that every device loading the library keeps
 * until exit.
 *   * limit: n * nw <= 2^21 words (16 MiB of keys); larger inputs return
 *     MH_EOVERFLOW and touch nothing;
 *   * the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress; again after the device's context is recreated);
 *     make that first call before any stream capture;
 *   * every call on a device shares the array and clears what must start at
 *     zero itself; calls that overlap on the GPU race and must be avoided;
 *   * every call with n >= 1 waits for `stream` before it returns (to read a
 *     status word, or after the single copy when n = 1).
 * Errors: MH_EINVAL (nw, key_bits, NULL, identical or misaligned buffers),
 * MH_EOVERFLOW,
 * MH_ETIMEOUT (a bounded look-back wait ran out), MH_EDEVICE. */
int mh_sort_keys_noalloc(const uint64_t* keys_in, uint64_t* keys_out, uint64_t n, int nw, int key_bits,
                         void* stream);

/* ------------------------------------------------------------ utilities */

const char* mh_strerror(int code);
const char* mh_last_error_message(const mh_ctx* ctx);

/* The context's stream (a cudaStream_t). */
void* mh_stream(const mh_ctx* ctx);

/* Bytes the context holds now, and the most it has held. */
void mh_memory(const mh_ctx* ctx, uint64_t* in_use, uint64_t* peak);
/* Return the device memory the context's own pool keeps cached to the
 * driver (after finishing the context's stream); no-op with allocator
 * callbacks.  Errors: MH_EINVAL, MH_EDEVICE. */
int mh_trim(mh_ctx* ctx);

/* Per-kernel launch statistics gathered while cfg.profile = 1 (or after
 * mh_set_profile(ctx, 1)).  Waits for the stream.  For index i in
 * [0, mh_profile_count()), writes the kernel's name (NUL-terminated, at most
 * name_cap bytes), its launch count, the sum of its CUDA-event durations in
 * milliseconds (events recorded on the context stream around each launch)
 * and the sum of its algorithmic bytes (the reads and writes the step must
 * do, e.g. 2 x key bytes per key for a radix pass; 0 where not accounted).
 * mh_profile_reset clears them.  Any output pointer may be NULL. */
int mh_profile_count(mh_ctx* ctx);
int mh_profile_get(mh_ctx* ctx, int i, char* name, int name_cap, uint64_t* launches, double* total_ms,
                   uint64_t* bytes);
void mh_profile_reset(mh_ctx* ctx);
void mh_set_profile(mh_ctx* ctx, int on);

#ifdef __cplusplus
}
#endif
#endif /* MH_H */
