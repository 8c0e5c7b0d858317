/*
 * zc.h -- C ABI of the GB300 error-bounded float codec and its collective
 * steps (gZCCL, arXiv 2308.05199).
 *
 * The library implements the GPU-side hot path of compression-accelerated
 * collectives: an error-bounded lossy compressor for FP32/BF16 buffers
 * (Sec. 3.3.2 adapts such a compressor for collectives), its decompressor, the
 * fused decompress -> sum -> recompress step each ring reduce-scatter round
 * runs on the received chunk (Sec. 3.2.3, 3.3.1 "GPU reduction kernel",
 * 3.3.3), and the per-destination pack of the compressed Scatter
 * (Sec. 3.3.4).  Every call is asynchronous on the given CUDA stream, takes
 * caller-owned device buffers, and never allocates: the paper's adapter
 * replaces per-call temporary allocations and unified-memory offset buffers
 * with one preallocated, reused device buffer (Sec. 3.3.2), here the
 * "workspace".
 *
 * Method (the paper does not print the compressor's internals; these are
 * this library's definitions, shared with its CPU oracle):
 *   q_i = the integer nearest to x_i / (2 eb), ties to even (exact);
 *   blocks of L = 16, 32, 64 or 128 elements, each delta-coded by a 1-D
 *   Lorenzo predictor (d_i = q_i - q_{i-1}, the block head predicted from 0);
 *   each block stored at a fixed bit width w = bit length of max |d|: a sign
 *   plane, then magnitude planes 0 .. w-1, L bits each;
 *   block payloads placed back to back at offsets given by a prefix sum of
 *   their sizes (computed on the device in one pass, decoupled look-back).
 * Reconstruction is x^ = fl32(q * 2eb): |x - q 2eb| <= eb exactly, and the
 * FP32 value adds at most half an FP32 ulp of x^ (BF16 output: half a BF16
 * ulp).
 *
 * Stream layout (little-endian, every stream a multiple of 16 bytes):
 *   [0,4) "ZCv1"  [4] dtype  [5] log2 L  [6] flags (bit 0: raw)  [7] 0
 *   [8,16) n  [16,20) eb (f32)  [20,24) nb = ceil(n / L)  [24,32) payload bytes
 *   [32, 32 + pad16(nb))          one width byte per block, zero padded
 *   [32 + pad16(nb), ... )        block payloads, zero padded to 16 bytes
 * A raw stream (flag bit 0) holds the n elements verbatim after the header.
 *
 * Error channels.
 *   - Argument errors are returned at once: a NULL pointer, a bad dtype or
 *     block size, a non-positive or non-finite bound, a workspace or output
 *     capacity that is too small for the header, a misaligned buffer.
 *     Nothing is launched then.
 *   - Data errors are only known on the device.  The first one is recorded in
 *     the workspace's status word (first error wins) and read back with
 *     zc_get_device_status().  Output content is unspecified after a data
 *     error, but no kernel ever writes outside [d_out, d_out + out_cap).
 *
 * Workspace.  One workspace per stream in flight (two calls that run at the
 * same time must not share one: Sec. 3.3.4 gives every stream its own
 * temporary buffers for the same reason).  Size it with zc_workspace_bytes(),
 * zero it once with zc_workspace_init(); after that no call needs it cleared
 * again: the look-back flags carry a launch generation number.
 *
 * Alignment.  Stream buffers (d_out, d_cmp*) must be 16-byte aligned; FP32
 * arrays 4-byte, BF16 arrays 2-byte aligned.
 */
#ifndef ZC_H
#define ZC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without the CUDA headers; 0 is the legacy default stream. */
typedef struct CUstream_st* zc_stream_t;

typedef enum {
    ZC_OK = 0,
    ZC_ERR_ARG = 1,       /* bad argument (returned at once)                  */
    ZC_ERR_RANGE = 2,     /* |x / 2eb| rounds beyond 2^22                      */
    ZC_ERR_NONFINITE = 3, /* NaN or Inf in the input                           */
    ZC_ERR_CAPACITY = 4,  /* output buffer too small                           */
    ZC_ERR_FORMAT = 5,    /* malformed or mismatched input stream              */
    ZC_ERR_TIMEOUT = 6,   /* a device-side wait gave up (see zc_set_wait_limit)*/
    ZC_ERR_CUDA = 7,      /* a CUDA runtime call failed                        */
    ZC_ERR_WORKSPACE = 8, /* workspace too small or not initialised            */
    ZC_ERR_BOUNDS = 9     /* bounds-checked build only: a kernel access fell
                             outside its buffer and was skipped (the status
                             detail is the offending offset)                  */
} zc_status;

typedef enum { ZC_F32 = 0, ZC_BF16 = 1 } zc_dtype;
typedef enum { ZC_EB_ABS = 0, ZC_EB_REL = 1 } zc_eb_mode;

#define ZC_HEADER_BYTES 32
#define ZC_MAX_WIDTH 24

/* Upper bound of the stream length for n elements at block size `block`
 * (every block at the largest width, 24): size d_out with it.  Sizing rule
 * only; no CUDA call. */
size_t zc_max_compressed_bytes(uint64_t n, int block);

/* Exact length of a raw stream of n elements of `dtype`. */
size_t zc_raw_stream_bytes(uint64_t n, int dtype);

/* Workspace bytes for calls on up to `n_total` elements spread over up to
 * `n_items` items (1 for single calls, P for batched ring steps and scatter
 * packs, M for batched compression).  Host-side arithmetic only.  Besides the
 * look-back records it holds the encoder CTAs' tile rings (staged payload of
 * the tiles in flight, at most 200 KB per CTA, up to 608 CTAs: at most
 * 124.5 MB); a smaller workspace still works, with fewer encoder CTAs. */
size_t zc_workspace_bytes(uint64_t n_total, int n_items);

/* Zero the workspace (cudaMemsetAsync) and stamp it as initialised.  Call
 * once after allocating it, on the stream that will use it. */
int zc_workspace_init(void* d_ws, size_t ws_bytes, zc_stream_t s);

/* Smallest and largest element of d_in[0..n) into d_minmax[0..1] (device
 * FP32).  Non-finite input sets ZC_ERR_NONFINITE.  Used to fix one relative
 * bound across several buffers (the ring takes one absolute bound for all its
 * steps). */
int zc_minmax(const void* d_in, uint64_t n, int dtype, float* d_minmax, void* d_ws,
              size_t ws_bytes, zc_stream_t s);

/* Compress d_in[0..n) (FP32 or BF16) into a stream at d_out.
 *   eb_mode ZC_EB_ABS: eb = eb_value.
 *   eb_mode ZC_EB_REL: eb = eb_value * (max - min) over the input in FP64
 *     (max(|max|, 1) when max == min), resolved on the device by one extra
 *     read of the input (value-range relative bound); the FP32 bound used is
 *     written into the stream header.
 *   block: 16, 32, 64 or 128.
 *   *d_out_bytes (device u64) receives the stream length.
 * The paper's Sec. 3.3.2 removes the offset buffer in unified memory and the
 * per-call allocations of the compressor it adapts; here offsets stay in the
 * workspace and nothing is read back to the host. */
int zc_compress(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value, int block,
                void* d_out, size_t out_cap, uint64_t* d_out_bytes, void* d_ws, size_t ws_bytes,
                zc_stream_t s);

/* Compression into the heads-apart stream format (header flag bit 1): every
 * block head q is stored in a fixed 24-bit little-endian two's-complement
 * field after the width bytes (3 nb bytes, zero padded to 16) and its own
 * delta is taken as 0, so a block's width covers only its in-block deltas.
 * Data on a large offset (a DC level far above eb) then costs 24 bits per
 * block instead of the offset's bit length on every element.  The paper's
 * blockwise Lorenzo predicts the block head from 0 (zc_compress); this
 * variant is this project's format extension, decoded by zc_decompress like
 * any stream.  Arguments as zc_compress; out_cap must hold at least the
 * header, width bytes and heads (32 + pad16(nb) + pad16(3 nb)), else
 * ZC_ERR_CAPACITY; zc_max_compressed_bytes_heads is the worst case.  Always
 * uses 8-chunk tiles. */
int zc_compress_heads(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value,
                      int block, void* d_out, size_t out_cap, uint64_t* d_out_bytes, void* d_ws,
                      size_t ws_bytes, zc_stream_t s);
size_t zc_max_compressed_bytes_heads(uint64_t n, int block);

/* Decompress a stream of n elements into d_out as FP32 or BF16 (RNE of the
 * FP32 reconstruction).  The stream's own header gives L and eb; a header
 * that does not match n, a width above 24 or a block that would read past
 * cmp_cap sets ZC_ERR_FORMAT.  Raw streams are copied (converted if
 * out_dtype differs). */
int zc_decompress(const void* d_cmp, size_t cmp_cap, void* d_out, uint64_t n, int out_dtype,
                  void* d_ws, size_t ws_bytes, zc_stream_t s);

/* One ring reduce-scatter step on one chunk (Sec. 3.2.3, 3.3.3): decode the
 * received stream d_cmp_in, add d_local (FP32, one rounding, decoded + local),
 * and re-encode the sum with the fixed absolute bound eb_abs at block size
 * `block` into d_cmp_out.  Without a received stream (d_cmp_in NULL) the
 * step is the ring's initial compression of d_local.  d_sum_out (nullable)
 * receives the FP32 sum; d_cmp_out may be NULL when only the sum is wanted
 * (the ring's last step).  Decompression, reduction and recompression run in
 * one kernel pass over the chunk (Sec. 3.3.1 moves the reduction to the GPU;
 * here it is fused with both codec passes). */
int zc_reduce_step(const void* d_cmp_in, size_t cmp_in_cap, const float* d_local, uint64_t n,
                   double eb_abs, int block, void* d_cmp_out, size_t out_cap,
                   uint64_t* d_out_bytes, float* d_sum_out, void* d_ws, size_t ws_bytes,
                   zc_stream_t s);

/* One ring step for all P simulated ranks in one launch.  Item r describes
 * rank r's chunk at this step (pointers as in zc_reduce_step, all device
 * pointers; cmp_in NULL for the initial compression). */
typedef struct {
    const void* cmp_in;      /* received stream or NULL                       */
    const float* local;      /* this rank's copy of the chunk (FP32)          */
    void* cmp_out;           /* output stream or NULL                         */
    float* sum_out;          /* FP32 sum or NULL                              */
    uint64_t* out_bytes;     /* device u64: output stream length              */
    uint64_t n;              /* chunk elements                                */
    uint64_t cmp_in_cap;     /* bytes readable at cmp_in                      */
    uint64_t out_cap;        /* bytes writable at cmp_out                     */
} zc_reduce_item;

/* A work-descriptor table in device memory, built once at set-up time (for
 * example one per ring step, for the whole ring) and launched any number of
 * times, also from a captured CUDA graph. */
typedef struct {
    int n_items;             /* descriptors in the table                      */
    int tile_chunks;         /* tile size the table was built for             */
    int block;               /* block size L                                  */
    int has_input;           /* some item decodes a received stream           */
    uint64_t total_tiles;    /* tiles of all items together                   */
    uint64_t total_chunks;   /* width-scan chunks of all items together       */
    const void* d_table;     /* the caller's device memory holding the table  */
} zc_plan;

/* Device bytes of a descriptor table for n_items items. */
size_t zc_plan_table_bytes(int n_items);

/* Build the table for one ring step over P ranks: validates every item,
 * splits the items into tiles and copies the table to d_table with a
 * synchronous cudaMemcpy (set-up time, not per step). */
int zc_plan_reduce(zc_plan* plan, int P, const zc_reduce_item* h_items, double eb_abs, int block,
                   void* d_table, size_t table_bytes);

/* Launch the planned ring step: all P ranks' decompress -> add -> recompress
 * in one kernel launch (the ring's per-round codec work of Sec. 3.2.3 for
 * every rank at once). */
int zc_reduce_step_batch(const zc_plan* plan, void* d_ws, size_t ws_bytes, zc_stream_t s);

/* Scatter pack (Sec. 3.3.4, compressed binomial-tree Scatter/Scatterv): the
 * root compresses segment p = d_in[h_displs[p] .. h_displs[p] + h_counts[p])
 * into a complete stream of its own, for p = 0 .. P-1, and the streams are
 * written back to back into d_out in one launch.  d_seg_off (device, P + 1
 * u64) receives the offset of each stream and the total length.  A relative
 * bound is resolved over all segments together.  P <= 1024. */
int zc_scatter_pack(const void* d_in, int dtype, int P, const uint64_t* h_counts,
                    const uint64_t* h_displs, int eb_mode, double eb_value, int block,
                    void* d_out, size_t out_cap, uint64_t* d_seg_off, void* d_ws,
                    size_t ws_bytes, zc_stream_t s);

/* ---- Batched compression: many messages, one launch ----------------------
 *
 * Sec. 3.2.2 observes that one compression launch per small message leaves
 * the GPU mostly idle, and Sec. 3.3.3 prices a collective's compression as
 * the cost of one compression times the number of them; this interface
 * compresses M messages of any sizes and either input
 * type, each with its own block size and absolute bound or stored raw, in
 * ONE persistent kernel launch.  Its CTAs take tiles of all messages from one
 * atomic ticket counter; every message becomes a complete, independent zc
 * stream (the format of zc_compress, raw streams with flag bit 0), and the
 * streams are written back to back (each a multiple of 16 bytes) into one
 * packed buffer.  d_msg_off (device, M + 1 u64) receives the start of every
 * stream and, in d_msg_off[M], the packed length.  Nothing is read back to
 * the host, so the launch can be captured in a CUDA graph (zc_graph_*). */
#define ZC_RAW 0             /* zc_message.block: store the message verbatim */
typedef struct {
    const void* in;          /* compression: the message's values (device)    */
    void* out;               /* decompression: where its values go (device)   */
    uint64_t n;              /* elements                                      */
    int dtype;               /* ZC_F32 or ZC_BF16: type of `in` (compression)
                                or of `out` (decompression)                   */
    int block;               /* 16, 32, 64 or 128, or ZC_RAW                  */
    double eb_abs;           /* absolute error bound (unused for ZC_RAW)      */
} zc_message;

/* A batch plan: a descriptor table in the caller's device memory, built once
 * at set-up time and launched any number of times. */
typedef struct {
    int n_msgs;
    int tile_chunks;         /* compression tile: chunks of 2048 elements     */
    int grid;                /* CTAs launched; 0 = as many as allowed         */
    int decompress;          /* 0: compression plan, 1: decompression plan    */
    int grouped;             /* 1: streams packed grouped by block size
                                (zc_batch_set_grouped); 0 after planning      */
    uint64_t total_tiles;    /* tiles of all messages together                */
    uint64_t total_chunks;   /* decompression: width-scan chunks              */
    const void* d_table;     /* the descriptor table (device)                 */
    void* d_packed;          /* the packed streams (device)                   */
    size_t packed_cap;       /* bytes at d_packed                             */
    uint64_t* d_msg_off;     /* M + 1 stream offsets (device)                 */
} zc_batch;

/* Device bytes of the descriptor table of a batch of n_msgs messages. */
size_t zc_batch_table_bytes(int n_msgs);

/* Largest packed length of the batch (every stream at its worst case);
 * 0 for an invalid message. */
size_t zc_batch_max_bytes(int n_msgs, const zc_message* h_msgs);

/* Plan the compression of h_msgs[0 .. n_msgs) into d_packed (16-byte
 * aligned).  tile_chunks: 4, 8, 16, or 0 for the current default
 * (zc_set_tile_chunks); grid: CTAs to launch (at most one per tile, per
 * ring of the workspace and 4 per SM), 0 = as many as allowed.  Validates
 * every message (ZC_ERR_ARG), checks that packed_cap holds at least every
 * header and width array (ZC_ERR_CAPACITY; the payload is checked on the
 * device), and copies the table to d_table with a synchronous cudaMemcpy. */
int zc_plan_compress_batch(zc_batch* plan, int n_msgs, const zc_message* h_msgs, int tile_chunks,
                           int grid, void* d_packed, size_t packed_cap, uint64_t* d_msg_off,
                           void* d_table, size_t table_bytes);

/* Launch a compression plan on s (one kernel).  Workspace: at least
 * zc_workspace_bytes(sum of n, n_msgs). */
int zc_compress_batch(const zc_batch* plan, void* d_ws, size_t ws_bytes, zc_stream_t s);

/* Plan the decompression of a packed buffer: stream i starts at
 * d_msg_off[i] (read on the device when the launch runs, so the offsets may
 * come from a compression launch earlier on the same stream) and decodes into
 * h_msgs[i].out as h_msgs[i].dtype; h_msgs[i].n must equal the stream's
 * element count (ZC_ERR_FORMAT on the device otherwise).  Offsets that are
 * not 16-byte aligned or lie outside packed_cap are format errors. */
int zc_plan_decompress_batch(zc_batch* plan, int n_msgs, const zc_message* h_msgs,
                             const void* d_packed, size_t packed_cap, const uint64_t* d_msg_off,
                             void* d_table, size_t table_bytes);

/* Plan the decompression of M streams at any device addresses (the
 * Allgather stage of a ring Allreduce, Sec. 3.3.3: every rank decodes the
 * chunks it does not own, one decompression per received chunk): stream i at
 * h_streams[i] (16-byte aligned, h_caps[i] readable bytes) decodes into
 * h_msgs[i].out as h_msgs[i].n elements of h_msgs[i].dtype (other fields
 * unused).  Launch with zc_decompress_batch. */
int zc_plan_decompress_streams(zc_batch* plan, int n_msgs, const void* const* h_streams,
                               const uint64_t* h_caps, const zc_message* h_msgs, void* d_table,
                               size_t table_bytes);

/* Launch a decompression plan on s (a width-scan and a decode kernel). */
int zc_decompress_batch(const zc_batch* plan, void* d_ws, size_t ws_bytes, zc_stream_t s);

/* Group a batch by block size (no counterpart in the paper).  A batch whose
 * neighbouring tiles use different block sizes makes the CTAs of one SM run
 * different encoder variants at once, which measured about twice as slow as
 * one block size throughout; grouped, a mixed batch runs at the mean of the
 * block sizes' own rates.  On a compression plan (grouped = 1), every
 * zc_compress_batch launch first orders the messages' tiles by block size
 * (raw, 16, 32, 64, 128; message order within a size) from the block sizes
 * in the device table at that moment -- so a selection written there by
 * zc_batch_select earlier on the same stream takes effect, also inside a
 * CUDA graph -- and packs the streams in that order: d_msg_off[i] is still
 * message i's start and d_msg_off[M] the packed length, but stream i need
 * not end where stream i + 1 starts (its header gives its length).  Three
 * small extra launches; the table's tile starts are rewritten on the device
 * (set again after every zc_plan_compress_batch, which clears the flag).  On
 * a decompression plan made with zc_plan_decompress_batch (grouped = 1), a
 * stream is bounded by d_msg_off[M] instead of d_msg_off[i + 1].  The streams
 * themselves are unchanged.  Host-only; ZC_ERR_ARG for a null plan, a value
 * other than 0 or 1, or a decompression plan without stream offsets. */
int zc_batch_set_grouped(zc_batch* plan, int grouped);

/* Autotuner for batched compression.  Times zc_compress_batch on the given
 * messages for every candidate tile size (4, 8, 16 chunks) and grid (1, 2 and
 * 4 CTAs per SM, and as many as allowed), and, with tune_block != 0, every
 * block size (16 .. 128, applied to all non-raw messages).  Each candidate
 * runs once untimed and `reps` times timed with CUDA events on s; its score
 * is the median time plus, for link_gbs > 0, the time to send the packed
 * bytes over a link of link_gbs GB/s (the end-to-end cost a compressed
 * collective pays).  Synchronous (set-up time).  Writes up to max_points
 * measured candidates to h_points (may be NULL), their number to *n_points
 * (may be NULL) and the best one to *best; leaves d_table planned with the
 * best candidate (call zc_plan_compress_batch again with best's settings to
 * rebuild it elsewhere).  The buffers must fit every candidate:
 * packed_cap >= zc_batch_max_bytes of the messages at the largest width. */
typedef struct {
    int block;               /* block size of the non-raw messages; 0 = as given */
    int tile_chunks;
    int grid;                /* 0 = as many CTAs as allowed                    */
    int status;              /* device status after the candidate's runs       */
    float ms;                /* median compression time                        */
    uint64_t packed_bytes;   /* packed length                                  */
    double score_ms;         /* ms + packed_bytes / link                       */
} zc_tune_point;

int zc_autotune_batch(int n_msgs, const zc_message* h_msgs, int tune_block, double link_gbs,
                      int reps, void* d_packed, size_t packed_cap, uint64_t* d_msg_off,
                      void* d_table, size_t table_bytes, void* d_ws, size_t ws_bytes,
                      zc_stream_t s, zc_tune_point* h_points, int max_points, int* n_points,
                      zc_tune_point* best);

/* ---- Per-chunk codec selection (statistics, MLP, choice) ------------------
 *
 * The paper runs one codec configuration per collective.  Sec. 3.2.2 shows
 * that a compression step's cost depends on the message, and Sec. 3.3.3
 * weighs compression cost against the bytes it saves on the link; the
 * selector below (an addition to the paper's method: it has no learned part)
 * makes that trade per chunk.  Every message of a compression plan is one
 * chunk (the selector's unit is 64 KiB; split longer buffers into messages of
 * that size).  The codec's arithmetic is unchanged: the selector only picks,
 * per message, the block size L in {16, 32, 64, 128} or raw storage. */
#define ZC_STATS 16
#define ZC_MLP_IN 16
#define ZC_MLP_HIDDEN 64
#define ZC_MLP_OUT 4
/* Parameters, FP32, in this order: W1[64][16], b1[64], W2[64][64], b2[64],
 * W3[4][64], b3[4] (row-major, W[out][in]). */
#define ZC_MLP_PARAMS 5508

/* Statistics of every message of a compression plan, 16 FP32 per message
 * into d_feat[n_msgs][16].  Sample: S = min(16, m) spans of 128 elements
 * (m = n / 128 full spans), span j at 128 * floor(j (m - 1) / (S - 1)); one
 * partial span when n < 128.  The sampled values are quantized exactly as the
 * codec does, with the message's bound.  Features:
 *   0..3  sampled bits per element at L = 16, 32, 64, 128 (the codec's
 *         (w + 1) L bits per block of width w > 0) + 8 / L + 256 / n;
 *   4     log2(1 + max q - min q);      5  log2(1 + mean |d|);
 *   6     log2(1 + max |d|);            7  fraction of d == 0;
 *   8     fraction of q == 0;           9  log2(1 + mean |q|);
 *   10    log2(1 + mean |d_i - d_{i-1}|);
 *   11    fraction of sign changes between consecutive d;
 *   12    mean bit length of |q| at L = 32 block heads / 24;
 *   13    standard deviation over spans of the span's L = 32 bits/element;
 *   14    raw bits per element / 32;    15 log2(n) / 16;
 * d = q_i - q_{i-1} within a span.  A message with no elements, no bound, or
 * a sampled value the codec cannot quantize gets a row of NaN.  One kernel,
 * one warp per message. */
int zc_batch_chunk_stats(const zc_batch* plan, float* d_feat, zc_stream_t s);

/* MLP forward: y[b] = W3 relu(W2 relu(W1 x'[b] + b1) + b2) + b3 with
 * x' = (x - mu) * inv_sd, d_norm = {mu[16], inv_sd[16]}; d_x[B][16] ->
 * d_y[B][4] (the four outputs: predicted log2 bits per element at L = 16 ..
 * 128 for the bits network, predicted log2 codec ns per input byte at L = 16
 * .. 128 for a time network of the same shape; the kernel is the same). */
int zc_mlp_forward(const float* d_params, const float* d_norm, const float* d_x, int B,
                   float* d_y, zc_stream_t s);

/* Scratch bytes of zc_mlp_grad for a minibatch of B rows. */
size_t zc_mlp_scratch_bytes(int B);

/* Gradient of the mean squared error sum((y - t)^2) / (4 B) over the
 * minibatch rows d_idx[0 .. B) of d_x / d_t (rows 0 .. B when d_idx is NULL)
 * into d_grad[ZC_MLP_PARAMS] (layout of the parameters); the loss into
 * *d_loss when d_loss is not NULL.  The ReLU derivative at 0 is 0.  Summation
 * order is fixed, so results are reproducible. */
int zc_mlp_grad(const float* d_params, const float* d_norm, const float* d_x, const float* d_t,
                const int* d_idx, int B, float* d_grad, float* d_loss, void* d_scratch,
                size_t scratch_bytes, zc_stream_t s);

/* Momentum SGD: v <- momentum v + g; p <- p - lr v (all ZC_MLP_PARAMS). */
int zc_mlp_sgd(float* d_params, float* d_vel, const float* d_grad, float lr, float momentum,
               zc_stream_t s);

/* Cost model of the selection: a message of n elements of s bytes costs,
 * coded at L_k with b bits per element, n s ns_per_byte[k] + (n b / 8) /
 * link_gbs ns, and raw, n s raw_ns_per_byte + (32 + n s) / link_gbs ns
 * (ns_per_byte: measured codec time, compression plus decompression, per
 * input byte; link_gbs in GB/s = bytes per ns).  With a time prediction
 * (zc_batch_select_timed) the message's own predicted ns per input byte
 * takes the place of ns_per_byte[k]. */
typedef struct {
    float link_gbs;
    float ns_per_byte[4];
    float raw_ns_per_byte;
    float judge_log2;        /* largest accepted |prediction - log2 estimate| */
    float judge_time_log2;   /* largest accepted |time prediction - log2 ns_per_byte[k]| */
} zc_select_cfg;

/* Choose every message's storage and write it into the plan's table (the
 * next zc_compress_batch of the plan uses it).  The heuristic: L = 32, or
 * raw when the cost with the sampled estimate (feature 1) is not below raw's.
 * With d_pred (zc_mlp_forward's output) the choice is the L of least cost
 * with bits 2^pred[k], or raw when that is cheaper -- unless a prediction is
 * not finite or the chosen L's prediction is more than judge_log2 from log2
 * of its sampled estimate (features 0..3): then the heuristic decides (a
 * fallback).  Messages planned raw stay raw.  d_choice[n_msgs] (nullable):
 * the block size, 0 for raw; d_counts[2] (nullable): fallbacks, raw
 * messages. */
int zc_batch_select(const zc_batch* plan, const float* d_feat, const float* d_pred,
                    const zc_select_cfg* cfg, int* d_choice, unsigned* d_counts, zc_stream_t s);

/* zc_batch_select with a second network's output as well: d_pred_time
 * [n_msgs][4] (zc_mlp_forward of a network trained on the codec's measured
 * times) holds the predicted log2 of the codec's ns per input byte
 * (compression plus decompression) of each message at L = 16 .. 128.  A
 * message's coded cost at L_k then uses 2^pred_time[k] in place of
 * cfg->ns_per_byte[k] -- unless that prediction is not finite or lies more
 * than cfg->judge_time_log2 from log2 ns_per_byte[k] (the measured batch-wide
 * rate judges it), where the batch-wide rate is kept.  The raw cost and the
 * bits side are as in zc_batch_select; d_pred_time == NULL is exactly
 * zc_batch_select.  The paper picks no per-chunk configuration (Sec. 3.2.2
 * measures that the codec's time depends on the message; Sec. 3.3.3 weighs
 * it against link time); this prediction is an addition to its method. */
int zc_batch_select_timed(const zc_batch* plan, const float* d_feat, const float* d_pred,
                          const float* d_pred_time, const zc_select_cfg* cfg, int* d_choice,
                          unsigned* d_counts, zc_stream_t s);

/* ---- CUDA graphs of zc calls ----------------------------------------------
 * Every zc launch function is asynchronous and reads nothing back, so a
 * sequence of them can be recorded once and replayed with one launch.
 * zc_graph_begin starts capturing s (a stream other than the legacy default
 * stream); the zc calls that follow on s are recorded, not run; zc_graph_end
 * stops the capture and instantiates the graph.  Make one ordinary call of
 * each entry point on the device before capturing it (the first call of a
 * kernel on each device sets its attributes), and build plans before the
 * capture (planning copies synchronously). */
typedef struct zc_graph_s* zc_graph;
int zc_graph_begin(zc_stream_t s);
int zc_graph_end(zc_stream_t s, zc_graph* g);
int zc_graph_launch(zc_graph g, zc_stream_t s);
void zc_graph_destroy(zc_graph g);

/* Compression for callers that may not allocate device memory (the paper has
 * no counterpart to this entry point).  Code on a collective's progress path
 * must not call cudaMalloc, which synchronises the whole device and would
 * stall the communication it serves; a plugin inside a framework that owns
 * all device memory through its own allocator has no way to obtain a
 * workspace.  This variant of zc_compress takes no workspace: its scratch
 * (look-back records, range partials, status word, the encoder's tile rings)
 * is one fixed 32 MiB device array inside this library, present on every GPU
 * that loads the library until the process exits; its rings allow about one
 * encoder CTA per SM.  It allocates nothing and calls no allocating
 * routine.
 *   - Arguments as zc_compress; n may not exceed ZC_NOALLOC_MAX_N (2^24
 *     elements), larger n returns ZC_ERR_ARG at once.
 *   - *d_status (device int, caller-owned) receives this call's device status
 *     (a zc_status, 0 = success) when the call has run on s.
 *   - The first call on a device sets the array up on that device (looks up
 *     its address, zeroes it on s); make that first call before any stream
 *     capture.
 *   - All calls share the one array: calls that overlap on the GPU (on
 *     different streams at the same time) race and corrupt each other's
 *     output; order them on one stream or with events. */
#define ZC_NOALLOC_MAX_N (1ull << 24)
int zc_compress_noalloc(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value,
                        int block, void* d_out, size_t out_cap, uint64_t* d_out_bytes,
                        int* d_status, zc_stream_t s);

/* Block until s is idle, then read the workspace status word (a zc_status)
 * and the index (element or tile) where the first error was seen. */
int zc_get_device_status(const void* d_ws, zc_stream_t s, int* status, uint64_t* detail);

/* Reset the status word (asynchronous on s). */
int zc_clear_device_status(void* d_ws, zc_stream_t s);

/* Every device-side wait (the look-back for a predecessor tile's offset) gives
 * up after this many nanoseconds, records ZC_ERR_TIMEOUT and returns.
 * Default 1 s; process-wide; applies to launches issued afterwards. */
void zc_set_wait_limit_ns(uint64_t ns);

/* Test hook: the tile with this index (within the next launches) does not
 * publish its offset, so that its successors' waits run out and report
 * ZC_ERR_TIMEOUT.  -1 (default) disables it. */
void zc_debug_withhold_tile(int64_t tile);

/* Tile size of the next encoder launches and plans: chunks of 2048 elements
 * per CTA tile (4, 8 or 16), or 0 (the default) to choose per launch: the
 * largest of 16 and 8 that is no larger than the launch's mean item and
 * still gives about 5/3 tiles per resident encoder CTA, else 4.  Larger
 * tiles shorten the chain of offsets between tiles and stage more bytes per
 * CTA in the workspace's tile rings (so the same workspace runs fewer CTAs
 * of them); small inputs keep more CTAs busy with small tiles.  Returns
 * ZC_ERR_ARG for other values.  Changes no stream byte. */
int zc_set_tile_chunks(int chunks);

/* Library version string. */
const char* zc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ZC_H */
