/*
 * lor.h -- C ABI of the GB300 longest-overlap-region library (liblor.so).
 *
 * Method: arXiv 1404.3448, "Solving The Longest Overlap Region Problem for
 * Noncoding DNA Sequences with GPU".  Section 3 states the problem (longest
 * common prefix of suffixes of the sequences and its positions in the suffix
 * array), builds the suffix array with DC3 (Steps 1-3, Tables 1-3), derives
 * the LCP array (LCP table), and answers LCP queries between arbitrary
 * suffixes as range minima (the lcp identity and the RMQ definition).
 * Section 4 (Algorithm 1) sorts DC3's keys with an LSD radix sort.
 *
 * Conventions shared by every call:
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *     are host pointers.  The caller owns and allocates every buffer; the
 *     library allocates no device memory and never frees caller memory.
 *   - Calls only enqueue work on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) and return without waiting, EXCEPT lor_build_sa, which
 *     reads one 4-byte count back per DC3 recursion level and per radix sort
 *     and therefore synchronises `stream` a few times per call.
 *   - The return value reports errors found on the host (null pointers, bad
 *     sizes, short workspace, CUDA launch errors).  Errors found by kernels
 *     (bad symbols, out-of-range indices in inputs, a bounded wait that ran
 *     out) are recorded in a per-device status word that lor_device_status()
 *     reads and clears.  No call traps, aborts or throws.
 *   - Indices are int32: texts hold at most LOR_MAX_N symbols.  The *64
 *     entry points (section "64-bit indices" below) take and return int64
 *     indices for texts of up to LOR_MAX_N64 symbols.
 */
#ifndef LOR_H
#define LOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lor_stream_t; /* same type as cudaStream_t */

/* Status codes. */
#define LOR_OK 0
#define LOR_ERR_INVALID_ARG (-1) /* null pointer, negative or zero size, bad nseq */
#define LOR_ERR_BAD_SYMBOL (-2)  /* input symbol outside ACGT/acgt, or text code out of [1, sigma) */
#define LOR_ERR_TOO_LARGE (-3)   /* n > LOR_MAX_N (LOR_MAX_N64 for the *64 calls), or an LCP past INT32_MAX */
#define LOR_ERR_WORKSPACE (-4)   /* workspace null or smaller than the *_workspace_size query */
#define LOR_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define LOR_ERR_TIMEOUT (-6)     /* a bounded inter-block wait ran out on the device */
#define LOR_ERR_BAD_INPUT (-7)   /* an input array holds an out-of-range index (SA, ISA, query) */
#define LOR_ERR_CANCELLED (-8)   /* server shut down before the request ran */

/* Largest supported text length (int32 indices with head-room for DC3's
 * dummy sample and padding). */
#define LOR_MAX_N 2147483000LL

/* Largest text length of the *64 entry points: positions are held as 32-bit
 * unsigned integers inside the library (every radix count, look-back value
 * and position fits), and a text this long already needs about 100 GB of
 * workspace. */
#define LOR_MAX_N64 4294901760LL

/* Largest number of sequences in one concatenated text (codes fit a byte). */
#define LOR_MAX_SEQ 250

/* Result of lor_longest_overlap (written to device memory). */
typedef struct {
    int32_t length; /* L: longest common region of two different sequences; 0 if none */
    int32_t rank;   /* smallest suffix-array index k >= 1 with SA[k-1], SA[k] in
                       different sequences and LCP[k] == L; -1 if L == 0 */
    int32_t seq_a;  /* lower sequence id of the pair at rank k; -1 if L == 0 */
    int32_t pos_a;  /* 0-based offset of that suffix inside sequence seq_a */
    int32_t seq_b;  /* higher sequence id of the pair at rank k */
    int32_t pos_b;  /* 0-based offset inside sequence seq_b */
    int32_t n_pos;  /* number of text positions whose length-L prefix also occurs
                       in another sequence (may exceed pos_cap) */
    int32_t reserved;
} lor_overlap;

/* ---------------------------------------------------------------------------
 * a1. Encode and concatenate (Section 3: the overlap of two or more
 * sequences is read off one suffix array; the separator scheme is this
 * library's reading, the paper states none).
 *
 * d_ascii    : device, the nseq sequences' ASCII bytes back to back
 *              (sum(h_lens) bytes; A/C/G/T in either case).
 * h_lens     : host, nseq lengths (each >= 0).
 * d_text     : device, receives n = sum(h_lens) + nseq codes: sequence i is
 *              followed by its terminator.  Codes: terminator of sequence i
 *              = nseq - i (1..nseq), A,C,G,T = nseq+1 .. nseq+4.  0 is
 *              reserved as padding and never written.  sigma = nseq + 5.
 * d_seq_starts: device int32[nseq + 1]: start of each sequence in d_text,
 *              d_seq_starts[nseq] = n.  May be NULL.
 * A symbol outside ACGT/acgt sets LOR_ERR_BAD_SYMBOL in the status word and is
 * stored as the code of A.  Returns LOR_ERR_INVALID_ARG for nseq outside
 * [1, LOR_MAX_SEQ], LOR_ERR_TOO_LARGE when n > LOR_MAX_N.
 * ------------------------------------------------------------------------- */
int lor_encode_concat(const uint8_t *d_ascii, const int64_t *h_lens, int32_t nseq,
                      uint8_t *d_text, int32_t *d_seq_starts, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * a2-a8. Suffix array by DC3 (Section 3, Steps 1-3; Tables 1-3), with the
 * sample and nonsample keys sorted by LSD radix sort (Section 4,
 * Algorithm 1).
 *
 * d_text : device uint8[n], codes in [1, sigma) (0 is reserved as padding);
 *          any text works, terminated (lor_encode_concat) or raw.  The end of
 *          the text compares smaller than every code.
 * sigma  : number of codes including 0 (2..256).
 * d_sa   : device int32[n], receives the suffix array: the start positions of
 *          the suffixes in increasing lexicographic order.
 * d_ws   : device workspace of at least lor_build_sa_workspace_size(n, sigma)
 *          bytes, 256-byte aligned; contents on entry are ignored.
 * A code outside [1, sigma) sets LOR_ERR_BAD_SYMBOL in the status word (the
 * output is then unspecified but every access stays in bounds).
 * Synchronises `stream` once per recursion level and per radix sort.
 * ------------------------------------------------------------------------- */
size_t lor_build_sa_workspace_size(int64_t n, int32_t sigma);
int lor_build_sa(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa,
                 void *d_ws, size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Suffix array without a workspace argument, for callers that cannot
 * allocate device memory (the paper has no counterpart; this is a library
 * convenience).  Same result and arguments as lor_build_sa.  Errors: the
 * argument checks of lor_build_sa come first (LOR_ERR_INVALID_ARG), then
 * n > LOR_NOALLOC_MAX_N returns LOR_ERR_TOO_LARGE before touching the
 * device; device-side errors as for lor_build_sa.  The scratch is one 32 MiB
 * array compiled into the library: every GPU that loads liblor holds it until
 * the process exits.  The first call on a device looks up the array's device
 * address and keeps it; do not call this entry point again after
 * cudaDeviceReset in the same process.  Like lor_build_sa it reads counts
 * back and synchronises `stream` during the call, so it cannot be captured
 * into a CUDA graph.  All calls share the array, so calls that can
 * overlap on the GPU race and must be serialised by the caller.  Allocates
 * nothing.
 * ------------------------------------------------------------------------- */
#define LOR_NOALLOC_MAX_N 262144LL
int lor_build_sa_noalloc(const uint8_t *d_text, int64_t n, int32_t sigma, int32_t *d_sa,
                         lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * a9. Inverse suffix array and LCP array (Section 3, LCP table; Kasai et al.,
 * cited there).  ISA[SA[k]] = k; LCP[0] = 0 and LCP[k] is the length of the
 * longest common prefix of the suffixes SA[k-1] and SA[k].
 *
 * d_text, n : as for lor_build_sa.   d_sa : device int32[n] suffix array.
 * d_isa     : device int32[n] output.  d_lcp : device int32[n] output.
 * d_ws      : device workspace of lor_lcp_workspace_size(n) bytes (about 25
 *             bytes per symbol), 256-byte aligned.
 * An SA entry outside [0, n) sets LOR_ERR_BAD_INPUT (and is skipped).
 * For n >= 2^20 synchronises `stream` once (the choice between the direct
 * comparison in rank order and Kasai's method for texts of long repeats is
 * read back); smaller texts take Kasai's method without a read-back.
 * ------------------------------------------------------------------------- */
size_t lor_lcp_workspace_size(int64_t n);
int lor_lcp(const uint8_t *d_text, const int32_t *d_sa, int64_t n, int32_t *d_isa,
            int32_t *d_lcp, void *d_ws, size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * a10. Longest overlap region (Section 3: the longest common prefix between
 * suffixes of the two sequences, with its positions in the suffix array).
 * L = max over k in [1, n) with seq(SA[k-1]) != seq(SA[k]) of LCP[k].
 *
 * d_seq_starts : device int32[nseq + 1] as written by lor_encode_concat.
 * d_out        : device, one lor_overlap (see the struct for the tie rule).
 * d_pos        : device int32[pos_cap] (may be NULL when pos_cap == 0):
 *                receives, sorted ascending, every text position p whose
 *                length-L prefix also occurs in another sequence (every
 *                member of a maximal rank run with adjacent LCP >= L that
 *                holds suffixes of two or more sequences).  Only the first
 *                pos_cap are written; d_out->n_pos holds the full count.
 * d_ws         : device workspace of lor_longest_overlap_workspace_size(n)
 *                bytes, 256-byte aligned.
 * ------------------------------------------------------------------------- */
size_t lor_longest_overlap_workspace_size(int64_t n);
int lor_longest_overlap(const int32_t *d_sa, const int32_t *d_lcp, int64_t n,
                        const int32_t *d_seq_starts, int32_t nseq, lor_overlap *d_out,
                        int32_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                        lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Longest overlap region of many sequence pairs (Section 3's problem, one
 * answer per pair; the batching is this library's).
 *
 * d_ascii   : device, the 2*npairs sequences' ASCII bytes back to back, pair
 *             p being sequences 2p and 2p+1.
 * h_lens    : host, 2*npairs lengths.
 * d_out     : device lor_overlap[npairs]: for every pair the record that
 *             lor_longest_overlap returns for that pair alone (sequence ids 0
 *             and 1, offsets inside the pair's sequences, rank inside the
 *             pair's own suffix array).
 * d_pos_off : device int64[npairs + 1]: pair p's positions occupy
 *             d_pos[d_pos_off[p] .. d_pos_off[p+1]), each an offset inside
 *             the pair's own text S1#S2$, ascending.
 * d_pos     : device int32[pos_cap]; positions beyond pos_cap are dropped
 *             (the offsets still count them).
 * d_ws      : lor_batch_workspace_size(h_lens, npairs) bytes, 256-byte aligned.
 * Pairs are processed in groups of up to 512 pairs and at most 2^28 symbols
 * (a single larger pair forms its own group); one DC3 suffix array over the
 * concatenated pair texts of a group is split into per-pair blocks.  A symbol
 * outside ACGT/acgt sets LOR_ERR_BAD_SYMBOL in the status word.  Synchronises `stream` a few times per group.
 * ------------------------------------------------------------------------- */
size_t lor_batch_workspace_size(const int64_t *h_lens, int32_t npairs);
int lor_batch_overlap(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs,
                      lor_overlap *d_out, int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap,
                      void *d_ws, size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched longest overlap replayed from one CUDA graph (no counterpart in
 * the paper; the batched pipeline of lor_batch_overlap captured once and
 * launched any number of times).
 *
 * lor_batch_graph_create captures the whole grouped pipeline for a fixed list
 * of pair lengths and fixed device buffers (d_ascii, d_out, d_pos_off, d_pos,
 * d_ws, the same meaning and layout as for lor_batch_overlap) into a CUDA
 * graph, without any host round trip inside: the suffix array of each group
 * sorts the level-0 sample by its 48-bit prefix and finishes the reduced
 * string by prefix doubling with every round enqueued up front (rounds whose
 * unresolved count, held on the device, is 0 do nothing); counts of later
 * stages stay on the device too.  Nothing runs on the device at creation.
 * lor_batch_graph_launch enqueues one replay on `stream`: it reads whatever
 * bases d_ascii holds at that time and writes every pair's record and
 * positions exactly as lor_batch_overlap does for them.
 * d_ws: lor_batch_graph_workspace_size(h_lens, npairs) bytes, 256-byte
 * aligned, used by nothing else while the graph exists.  Replays of one graph
 * must not overlap on the device (they share d_ws).  The graph owns a little
 * pinned host memory, freed by lor_batch_graph_destroy.
 * Returns LOR_ERR_CUDA when capture or instantiation fails.
 * ------------------------------------------------------------------------- */
typedef struct lor_batch_graph lor_batch_graph;
size_t lor_batch_graph_workspace_size(const int64_t *h_lens, int32_t npairs);
int lor_batch_graph_create(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs,
                           lor_overlap *d_out, int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap,
                           void *d_ws, size_t ws_bytes, lor_batch_graph **out);
int lor_batch_graph_launch(lor_batch_graph *g, lor_stream_t stream);
/* Kernels one replay launches (for launch accounting). */
int64_t lor_batch_graph_kernels(const lor_batch_graph *g);
int lor_batch_graph_destroy(lor_batch_graph *g);

/* ---------------------------------------------------------------------------
 * a11/a12 in linear space (Section 3: the same range minimum, stored in
 * O(n) words; the paper's own linear-space RMQ is a +-1 RMQ over a Cartesian
 * tree, this is a block decomposition).
 * The LCP array is cut into blocks of 32 entries; the table is a sparse
 * table over the block minima: levels = floor(log2 nb) + 1 rows of
 * stride = nb rounded up to 64 entries, nb = ceil(n / 32), with
 * table[j*stride + b] = min(blockmin[b .. min(b + 2^j, nb) - 1]) and
 * blockmin[b] = min(lcp[32b .. min(32b + 32, n) - 1]).  d_table must be
 * 256-byte aligned and hold lor_rmq_block_table_elems(n) int32 entries
 * (n / 32 * (log2 n - 4) words, under a tenth of the sparse table at any n
 * above 2^16).  lor_rmq_block_table_elems and lor_rmq_block_build accept n up
 * to LOR_MAX_N64 (the table of a 64-bit text; query it with
 * lor_rmq_block_query64).
 * lor_rmq_block_query answers exactly what lor_rmq_query answers (same
 * arguments, same errors) and also reads d_lcp: the partial blocks at both
 * ends of a rank range are scanned in the LCP array, the whole blocks between
 * them read from the table.
 * ------------------------------------------------------------------------- */
int64_t lor_rmq_block_table_elems(int64_t n);
int lor_rmq_block_build(const int32_t *d_lcp, int64_t n, int32_t *d_table, int64_t table_elems,
                        lor_stream_t stream);
int lor_rmq_block_query(const int32_t *d_table, const int32_t *d_lcp, const int32_t *d_isa, int64_t n,
                        const int32_t *d_p, const int32_t *d_q, int64_t nq, int32_t *d_out,
                        lor_stream_t stream);
/* The index form of the RMQ (Section 3: RMQ returns the position of the
 * minimum): for suffixes p[i] != q[i] with ranks r1 < r2, d_val[i] = the
 * minimum of lcp(r1, r2] (the LCP of the two suffixes) and d_arg[i] = the
 * leftmost rank k in (r1, r2] where it occurs; p[i] == q[i] gives
 * d_val[i] = n - p[i], d_arg[i] = -1.  Same table, inputs and errors as
 * lor_rmq_block_query (a bad position yields -1 in both outputs). */
int lor_rmq_block_argmin(const int32_t *d_table, const int32_t *d_lcp, const int32_t *d_isa, int64_t n,
                         const int32_t *d_p, const int32_t *d_q, int64_t nq, int32_t *d_val, int32_t *d_arg,
                         lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * The K longest maximal overlaps (extends a10 from the maximum to the K
 * largest values of the same quantity).
 * A candidate is a rank k in [1, n) whose adjacent suffixes a = SA[k-1],
 * b = SA[k] start in different sequences, with LCP[k] > 0, and that is
 * left-maximal: a == 0, b == 0, or text[a-1] != text[b-1] (so each shared
 * region is reported once, not once per shifted copy).  d_out[0 .. *d_count)
 * receives the min(K, candidates) largest by (LCP desc, rank asc) as overlap
 * records (length, rank, seq_a/pos_a on the lower sequence id, seq_b/pos_b;
 * n_pos = 0).  Inputs as for lor_longest_overlap plus the text; d_count is
 * one device int32.  1 <= K <= LOR_TOPK_MAX.  d_ws:
 * lor_topk_overlaps_workspace_size(n) bytes, 256-byte aligned.
 * ------------------------------------------------------------------------- */
#define LOR_TOPK_MAX 65536
size_t lor_topk_overlaps_workspace_size(int64_t n);
int lor_topk_overlaps(const uint8_t *d_text, const int32_t *d_sa, const int32_t *d_lcp, int64_t n,
                      const int32_t *d_seq_starts, int32_t nseq, int32_t K, lor_overlap *d_out,
                      int32_t *d_count, void *d_ws, size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * One reference against many query sequences (the paper's experiments take
 * 512 .. 2,097,152 query sequences against a reference; Section 3 defines
 * the overlap through common prefixes of suffixes).
 *
 * For each query Q_i: the longest substring it shares with the reference R
 * (length), the smallest offset in Q_i where a substring of that length
 * shared with R starts (query_pos), and the smallest offset in R where
 * Q_i[query_pos, query_pos + length) occurs (ref_pos).  length 0 (no common
 * base, or an empty sequence) gives query_pos = ref_pos = -1.
 * d_ref: ASCII ACGT/acgt, ref_len bytes (device).  d_queries: the queries'
 * ASCII bases back to back (device), lengths h_q_lens[0 .. nq) (host).
 * d_out: device lor_mq_hit[nq].  d_ws: lor_multi_query_workspace_size bytes,
 * 256-byte aligned.  One suffix array is built over R 1 Q_1 2 Q_2 2 ...
 * (code 1 ends the reference, code 2 every query), so the work is that of
 * one text of ref_len + sum(lengths) + nq + 1 symbols, not one per query.
 * nq <= LOR_MQ_MAX_QUERIES and the text at most LOR_MAX_N symbols, else
 * LOR_ERR_TOO_LARGE.  A symbol outside ACGT/acgt sets LOR_ERR_BAD_SYMBOL in
 * the status word.
 * ------------------------------------------------------------------------- */
#define LOR_MQ_MAX_QUERIES 4194304
typedef struct {
    int32_t length;
    int32_t query_pos;
    int32_t ref_pos;
    int32_t reserved;
} lor_mq_hit;
size_t lor_multi_query_workspace_size(int64_t ref_len, const int64_t *h_q_lens, int32_t nq);
int lor_multi_query_overlap(const uint8_t *d_ref, int64_t ref_len, const uint8_t *d_queries,
                            const int64_t *h_q_lens, int32_t nq, lor_mq_hit *d_out, void *d_ws,
                            size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Launch parameters and their autotuner (no counterpart in the paper).
 *
 * Every value gives the same results; only the speed differs.  The
 * configuration is process-wide: set it before work is enqueued from other
 * threads.  A call reads it when it starts; a CUDA graph keeps the values it
 * was captured with.
 *   digit_bits      radix digit width of every sort pass, 5..8 (default 8)
 *   level0_key_bits width of the level-0 sample keys, 24..60 (default 48): DC3
 *                   level 0 names the longest prefix whose key in base
 *                   (largest code + 1) fits it, so wider keys cost radix passes
 *                   and leave fewer repeated names for the later rounds (texts
 *                   that take 2-bit keys, see lor_dc3_route_set, and the
 *                   batched pipeline's graph-captured route excepted)
 *   sort_items_64   keys per thread of a sort pass over 64-bit keys: 8, 12 or 16 (12)
 *   sort_items_32   keys per thread over 32-bit keys: 12 or 16 (16)
 *   merge_items     merged suffixes per thread of the Step-3 merge: 2, 4 or 8
 *                   (512-, 256- or 128-thread blocks); default 4
 * lor_tune_set returns LOR_ERR_INVALID_ARG for a value out of range (and
 * changes nothing).
 *
 * lor_autotune_batch times lor_batch_overlap on the caller's pairs (the same
 * arguments, buffers and workspace as lor_batch_overlap) for candidate values,
 * one parameter at a time in the order above, starting from the current
 * configuration and keeping a change only when it is faster: every candidate
 * runs once untimed and then `reps` times (1..100) between CUDA events on
 * `stream`.  On return the fastest configuration found is set and copied to
 * *best, and *best_ms holds its time per run.  Synchronises `stream`.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t digit_bits;
    int32_t level0_key_bits;
    int32_t sort_items_64;
    int32_t sort_items_32;
    int32_t merge_items;
} lor_tune;
void lor_tune_default(lor_tune *cfg);
int lor_tune_get(lor_tune *cfg);
int lor_tune_set(const lor_tune *cfg);
int lor_autotune_batch(const uint8_t *d_ascii, const int64_t *h_lens, int32_t npairs, lor_overlap *d_out,
                       int64_t *d_pos_off, int32_t *d_pos, int64_t pos_cap, void *d_ws, size_t ws_bytes,
                       int32_t reps, lor_stream_t stream, lor_tune *best, double *best_ms);

/* ---------------------------------------------------------------------------
 * a11. Sparse table over the LCP array for range-minimum queries (Section 3:
 * RMQ definition; the LCP of arbitrary suffixes is a range minimum).
 * Layout: level-major, levels = floor(log2 n) + 1 rows of
 * stride = lor_rmq_row_stride(n) entries (n rounded up to a multiple of 64);
 * table[j*stride + i] = min(lcp[i .. min(i + 2^j, n) - 1]) for i < n (the
 * padding entries are unspecified).  d_table must be 256-byte aligned and
 * hold at least lor_rmq_table_elems(n) = levels * stride int32 entries.
 * ------------------------------------------------------------------------- */
int64_t lor_rmq_row_stride(int64_t n);
int64_t lor_rmq_table_elems(int64_t n);
int lor_rmq_build(const int32_t *d_lcp, int64_t n, int32_t *d_table, int64_t table_elems,
                  lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * a12. LCP of arbitrary suffix pairs (Section 3: lcp(S_p, S_q) = min of the
 * adjacent LCPs strictly between their ranks, through the RMQ).
 * out[i] = length of the longest common prefix of suffixes p[i] and q[i]
 * (n - p[i] when p[i] == q[i]).  All arrays device, int32[nq].
 * A p or q outside [0, n) sets LOR_ERR_BAD_INPUT and yields -1 for that query.
 * ------------------------------------------------------------------------- */
int lor_rmq_query(const int32_t *d_table, const int32_t *d_isa, int64_t n, const int32_t *d_p,
                  const int32_t *d_q, int64_t nq, int32_t *d_out, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Request server: pair requests arrive one by one; each gets the longest
 * overlap region of its pair (Section 3's problem) and then answers LCP
 * queries between arbitrary suffixes of its own text S1#S2$ (Section 3: the
 * LCP of two suffixes through the RMQ over the LCP array) while its state
 * stays resident.  The serving loop has no counterpart in the paper.
 *
 * lor_server_create reserves hbm_budget_bytes of device memory on the current
 * device (one allocation; the server allocates nothing else on the device
 * afterwards except its small query buffers) and starts `workers` threads,
 * each with its own non-blocking stream.  A free worker takes the oldest
 * waiting requests (at most max_batch_pairs pairs and max_batch_symbols text
 * symbols) as one batch, admits it when the batch's workspace and resident
 * state fit in the reserved memory (otherwise it waits until a batch finishes
 * or a request is released; requests are admitted in arrival order), copies
 * the pairs to the device and runs the grouped pipeline of lor_batch_overlap
 * on them.  Batches of different workers run on the device at once.  After a
 * batch, its workspace is returned to the reservation; the batch's ISA, its
 * LCP array and a block table over it (the linear-space RMQ of
 * lor_rmq_block_build, about 10.6 bytes per symbol in all) stay resident until every request of the
 * batch has been released.
 *
 * Results do not depend on how requests are batched: a request's record,
 * positions and query answers equal those of lor_longest_overlap and
 * lor_rmq_query run on its pair alone.
 *
 * Ownership: the host sequences passed to lor_server_submit must stay valid
 * and unchanged until the request's result has been returned by
 * lor_server_poll (pinned memory makes the copies faster).  The positions
 * pointer of a result is owned by the server and valid until
 * lor_server_release.  Times are seconds on a monotonic clock whose zero is
 * the server's creation.  All functions are thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct lor_server lor_server;

typedef struct {
    size_t hbm_budget_bytes;   /* device memory reserved for batches and resident state */
    int32_t workers;           /* concurrent batches, 1 .. 8 */
    int32_t max_batch_pairs;   /* 1 .. 512 */
    int64_t max_batch_symbols; /* text symbols per batch, 1 .. 2^28 (a single larger pair still runs alone) */
} lor_server_config;

typedef struct {
    int64_t id;          /* returned by lor_server_submit */
    uint64_t tag;        /* caller's tag, passed through */
    int32_t status;      /* LOR_OK, or the error that ended the request's batch */
    int32_t batch_pairs; /* pairs in the batch the request ran in */
    lor_overlap ov;      /* as lor_longest_overlap on the pair alone */
    const int32_t *positions; /* ov.n_pos offsets in S1#S2$, ascending (server-owned) */
    double t_submit, t_admit, t_done; /* submit, batch admitted, result ready */
} lor_served;

typedef struct {
    int64_t submitted, completed, released, batches, pairs, bases;
    int64_t admission_waits;   /* times a free worker waited for reserved memory */
    int64_t queries;           /* LCP queries answered */
    size_t reserved_bytes, in_use_bytes, peak_bytes;
    int32_t pending, in_flight;
} lor_server_stats;

/* Device bytes one batch of the given pairs takes from the reservation while
 * it runs (the first value) and afterwards until released (*h_resident). */
size_t lor_server_batch_bytes(const int64_t *h_lens, int32_t npairs, size_t *h_resident);
int lor_server_create(const lor_server_config *cfg, lor_server **out);
/* Queues one pair; *out_id receives its id.  LOR_ERR_TOO_LARGE if the pair
 * alone cannot fit in the reservation; LOR_ERR_INVALID_ARG for null pointers
 * with nonzero length or negative lengths. */
int lor_server_submit(lor_server *srv, const uint8_t *h_a, int64_t len_a, const uint8_t *h_b,
                      int64_t len_b, uint64_t tag, int64_t *out_id);
/* Moves up to cap finished requests into out[], waiting up to timeout_ms for
 * the first; returns how many (or a negative status). */
int lor_server_poll(lor_server *srv, lor_served *out, int32_t cap, int32_t timeout_ms);
/* LCP of suffixes h_p[i] and h_q[i] of request id's text S1#S2$ (as
 * lor_rmq_query on the pair alone), for a request whose result was polled
 * and not yet released.  Host arrays of nq entries; synchronous.
 * LOR_ERR_INVALID_ARG for an unknown id or a suffix outside the text. */
int lor_server_query(lor_server *srv, int64_t id, const int32_t *h_p, const int32_t *h_q, int32_t nq,
                     int32_t *h_out);
/* Drops a polled request's result and resident state. */
int lor_server_release(lor_server *srv, int64_t id);
int lor_server_stats_get(lor_server *srv, lor_server_stats *out);
/* Seconds on the server's clock (the clock of the t_* fields). */
double lor_server_now(lor_server *srv);
/* Stops the workers after their current batches, drops waiting and unreleased
 * requests and frees everything (result pointers become invalid).  Submits
 * racing with it return LOR_ERR_CANCELLED. */
int lor_server_destroy(lor_server *srv);

/* ---------------------------------------------------------------------------
 * The radix sort of Section 4 (Algorithm 1) as a standalone primitive:
 * stable LSD sort of m (key, value) pairs by the low key_bits bits of the
 * keys, in place.  d_keys uint64[m], d_vals uint32[m]; d_ws of
 * lor_radix_sort_workspace_size(m) bytes.  Synchronises `stream` once.
 * ------------------------------------------------------------------------- */
size_t lor_radix_sort_workspace_size(int64_t m);
int lor_radix_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, int64_t m, int32_t key_bits,
                         void *d_ws, size_t ws_bytes, lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * 64-bit indices: the path a1-a12 for texts longer than LOR_MAX_N, up to
 * LOR_MAX_N64 symbols (chromosome-scale concatenations).  Indices that can
 * pass 2^31 (text positions, suffix-array ranks, sequence starts, offsets and
 * counts) are int64; LCP values stay int32 (an LCP above INT32_MAX sets
 * LOR_ERR_TOO_LARGE in the status word).  Any n >= 1 is accepted, so the
 * calls can be checked on small texts.  Errors as for the int32 calls, with
 * LOR_MAX_N64 in place of LOR_MAX_N.
 * ------------------------------------------------------------------------- */

/* a1: as lor_encode_concat; d_seq_starts is device int64[nseq + 1]. */
int lor_encode_concat64(const uint8_t *d_ascii, const int64_t *h_lens, int32_t nseq, uint8_t *d_text,
                        int64_t *d_seq_starts, lor_stream_t stream);

/* a2-a8: the suffix array (the order of Section 3, Tables 1-3) as int64[n].
 * Built by prefix doubling over all suffixes (the reduced-string finisher of
 * lor_build_sa, started on the text): one LSD radix sort of every suffix's
 * first floor(64 / b) codes (b = bits of sigma - 1), then rounds that sort
 * only the still-tied suffixes by the rank of the suffix h symbols on,
 * h doubling each round.  Same text convention and errors as lor_build_sa.
 * d_ws: lor_build_sa64_workspace_size(n, sigma) bytes (about 44 n),
 * 256-byte aligned.  Synchronises `stream` once per round and per radix sort. */
size_t lor_build_sa64_workspace_size(int64_t n, int32_t sigma);
int lor_build_sa64(const uint8_t *d_text, int64_t n, int32_t sigma, int64_t *d_sa, void *d_ws, size_t ws_bytes,
                   lor_stream_t stream);

/* a9: ISA (int64[n]) and LCP (int32[n]) from an int64 suffix array, as
 * lor_lcp.  d_ws: lor_lcp64_workspace_size(n) bytes (about 29 n). */
size_t lor_lcp64_workspace_size(int64_t n);
int lor_lcp64(const uint8_t *d_text, const int64_t *d_sa, int64_t n, int64_t *d_isa, int32_t *d_lcp, void *d_ws,
              size_t ws_bytes, lor_stream_t stream);

/* a10: the longest overlap record with int64 rank, offsets and count, and the
 * sorted positions as int64; otherwise as lor_longest_overlap (same tie rule,
 * same position set).  d_seq_starts: device int64[nseq + 1].
 * d_ws: lor_longest_overlap64_workspace_size(n) bytes. */
typedef struct {
    int32_t length;   /* L; 0 if none */
    int32_t seq_a;    /* lower sequence id of the pair at rank k; -1 if L == 0 */
    int32_t seq_b;    /* higher sequence id; -1 if L == 0 */
    int32_t reserved;
    int64_t rank;     /* k; -1 if L == 0 */
    int64_t pos_a;    /* offset inside seq_a; -1 if L == 0 */
    int64_t pos_b;    /* offset inside seq_b; -1 if L == 0 */
    int64_t n_pos;    /* number of positions (may exceed pos_cap) */
} lor_overlap64;
size_t lor_longest_overlap64_workspace_size(int64_t n);
int lor_longest_overlap64(const int64_t *d_sa, const int32_t *d_lcp, int64_t n, const int64_t *d_seq_starts,
                          int32_t nseq, lor_overlap64 *d_out, int64_t *d_pos, int64_t pos_cap, void *d_ws,
                          size_t ws_bytes, lor_stream_t stream);

/* a12 on the block table of a 64-bit text (lor_rmq_block_build with the
 * int32 LCP array): int64 ISA, query positions and answers (p == q answers
 * the suffix length n - p); otherwise as lor_rmq_block_query. */
int lor_rmq_block_query64(const int32_t *d_table, const int32_t *d_lcp, const int64_t *d_isa, int64_t n,
                          const int64_t *d_p, const int64_t *d_q, int64_t nq, int64_t *d_out,
                          lor_stream_t stream);

/* ---------------------------------------------------------------------------
 * Status, diagnostics and instrumentation (no counterpart in the paper).
 * ------------------------------------------------------------------------- */
/* Synchronise `stream`, then return and clear the first device-side error
 * recorded on the current device since the last call (LOR_OK if none). */
int lor_device_status(lor_stream_t stream);
const char *lor_status_string(int status);

/* Number of kernels this library has launched in this process. */
uint64_t lor_launch_count(void);

/* Per-level trace of the most recent lor_build_sa call on the calling thread:
 * fills up to cap entries of level length n_l, distinct names found at that
 * level, key bits of the sample keys (33 for level 0's 2-bit keys: 32 bits
 * and the exception bit), how the sample was ordered (0 radix
 * sort, 1 dense naming table, 2 the parent level's order, 3 prefix doubling
 * of the reduced string in place of a DC3 level) and how many samples shared
 * their first symbol (strategy 2) or their name (strategy 3); any pointer
 * may be NULL.
 * Returns the number of levels. */
int lor_last_dc3_trace(int64_t *h_n, int64_t *h_names, int32_t *h_key_bits, int32_t *h_strategy,
                       int64_t *h_dups, int32_t cap);

/* Kernel timing: when enabled, every launch records a CUDA event pair on its
 * stream together with the algorithmic bytes it moves.  lor_profile_read
 * synchronises those events and returns, for one kernel kind, the launch
 * count, summed device milliseconds and summed algorithmic bytes. */
int lor_profile_enable(int on);
int lor_profile_reset(void);
int lor_profile_kinds(void);
const char *lor_profile_kind_name(int kind);
int lor_profile_read(int kind, int64_t *h_launches, double *h_ms, double *h_bytes);

/* ---------------------------------------------------------------------------
 * Route controls of the suffix array (DC3, Section 3 Steps 1-3).  They change
 * how lor_build_sa orders its samples, never its result, and exist so that
 * tests can force every route and a measurement can time the plain
 * recursion.  Process-wide; read once at the start of each lor_build_sa call
 * (also inside the batched, served and no-workspace calls).
 *   level0_symbols: symbols named at level 0.  0 = automatic: for a text whose
 *                   symbols are the four largest codes but for at most 4096
 *                   sample windows (DNA with its separators), the first 16
 *                   symbols at 2 bits each; otherwise as 1.  1 = the longest
 *                   prefix whose key, in base sigma, fits the tuned level-0
 *                   key width.  3..64 = that many symbols, in base sigma.
 *   strategy      : 0 = pick per level (dense table, parent order or sort),
 *                   1 = radix sort at every level.
 *   doubling      : 0 = never (recurse while names repeat, as the paper
 *                   does), 1 = finish by prefix doubling once names are almost
 *                   unique (default), 2 = whenever names repeat.
 * lor_dc3_route_set(0, 0, 1) restores the defaults.  Returns
 * LOR_ERR_INVALID_ARG (and changes nothing) for a value out of range.
 * ------------------------------------------------------------------------- */
int lor_dc3_route_set(int32_t level0_symbols, int32_t strategy, int32_t doubling);
int lor_dc3_route_get(int32_t *level0_symbols, int32_t *strategy, int32_t *doubling);

/* ---------------------------------------------------------------------------
 * Test-only control of the bounded waits (no counterpart in the paper).
 * Every inter-block wait of every kernel gives up after limit_ns nanoseconds
 * (0 = the default of 2 s, also the maximum) and records LOR_ERR_TIMEOUT.
 * starve_first_tile = 1 makes the first tile of every LSD radix pass withhold
 * its look-back descriptor, so that the tile after it must wait until the
 * limit runs out: a way to exercise the timeout path without a fault.  The
 * results of a call made in that state are unspecified (every access stays
 * in bounds).  lor_test_set_wait(0, 0) restores normal operation.  Applies
 * to work launched after the call; synchronous.
 * ------------------------------------------------------------------------- */
int lor_test_set_wait(uint64_t limit_ns, int32_t starve_first_tile);

#ifdef __cplusplus
}
#endif

#endif /* LOR_H */
