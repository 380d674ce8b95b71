/*
 * pmklc.h — C ABI of libpmklc.so, a GB300 (sm_103a) implementation of the
 * per-block learned-compression loop of PMKLC (Sun et al., arXiv 2507.12805).
 *
 * Conventions for every entry point
 *   - Return 0 (PMKLC_OK) on success or a negative PMKLC_E* code; nothing
 *     aborts, traps or exits.  pmklc_strerror() names a code.
 *   - "d_" arguments are device pointers (CUDA global memory of the current
 *     device), everything else is host memory.  Inputs are read-only and stay
 *     owned by the caller.  Buffers returned through `uint8_t **` etc. are
 *     allocated by the library and released with pmklc_free().
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     is ordered on it; calls that return host results synchronise it.
 *   - Sizes are element counts unless the name says bytes.
 *   - Token arrays are uint16 (k <= 8, so 4^k <= 65536 symbols).
 *   - One process drives one CUDA device: the GEMM kernels' shared-memory
 *     opt-in is made once per process.  Calls from several host threads on
 *     their own streams share only mutex-guarded caches, the per-thread
 *     statistics and the process-wide profiler (enable it around one call at a
 *     time); concurrent calls are not tested, and pmklc_crc32_noalloc's scratch
 *     must be serialised by the caller.
 *   - A model's parameters are one FP32 array in the layout
 *         Emb[A][E] | W1t[H][t*E] | b1[H] | W2[H][A] | b2[A]     (A = 4^k)
 *     (row-major; W1 is stored transposed, row j holding the weights into
 *     hidden unit j), see pmklc_model_count(); a BiGRU static predictor's
 *     layout is given at pmklc_predict_bigru().
 */
#ifndef PMKLC_H
#define PMKLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMKLC_ABI_VERSION 4

/* error codes */
#define PMKLC_OK 0
#define PMKLC_EINVAL (-1)   /* bad argument, non-ACGT byte, s > k, k > 8, ... */
#define PMKLC_ENOMEM (-2)   /* host or device allocation failed */
#define PMKLC_ECUDA (-3)    /* a CUDA runtime call failed */
#define PMKLC_ECORRUPT (-4) /* malformed container, checksum or token mismatch */
#define PMKLC_EMODEL (-5)   /* static weights differ from the ones in the container */
#define PMKLC_ETIMEOUT (-6) /* a bounded device wait expired */
#define PMKLC_ENOSPC (-7)   /* caller's output buffer too small */

/* precision forms */
#define PMKLC_FP32_PLAIN 0
#define PMKLC_BF16_BATCHED 1
/* BF16 batched, with the frozen static predictor in FP8 (E4M3 weights with one scale per
   channel, E4M3 activations): see pmklc_quantize_static_fp8 */
#define PMKLC_BF16_FP8STATIC 2
/* BF16 batched, with the frozen static predictor's embedding and hidden layer in FP8 (E4M3
   embedding, E4M3 W1 with one scale per hidden unit; h written in BF16) and its logits layer in
   BF16: the logits layer's E4M3 weights carry almost all of PMKLC_BF16_FP8STATIC's loss */
#define PMKLC_BF16_FP8HIDDEN 3
#define PMKLC_UPDATE_AUTO 0
#define PMKLC_UPDATE_STREAM 1
#define PMKLC_UPDATE_FUSED 2
/* optimisers */
#define PMKLC_ADAM 0
#define PMKLC_SGD 1
/* step-wise model passing schedules */
#define PMKLC_SMP_NONE 0
#define PMKLC_SMP_CHAIN 1
#define PMKLC_SMP_TREE 2

/*
 * Model and run configuration (paper §4.2 AMKLCF, §4.3 DC + SMP, §5.1.4
 * parameters).  struct_size must be sizeof(pmklc_model_cfg).
 */
typedef struct {
  uint32_t struct_size;
  uint32_t s, k;               /* (s,k)-mer step and window, 1 <= s <= k <= 8 (§4.1) */
  uint32_t use_static;         /* S0 of Eq. (1): mix in the frozen static predictor */
  uint32_t emb_s, ctx_s, hid_s;/* static predictor: embedding E, context t, hidden H */
  uint32_t emb_d, ctx_d, hid_d;/* dynamic predictor (trained online, §4.2.4) */
  uint32_t lanes_per_block;    /* M: parallel sub-streams per block (bs, §5.8); 0 = default */
  uint32_t precision;          /* PMKLC_FP32_PLAIN, PMKLC_BF16_BATCHED, PMKLC_BF16_FP8STATIC or PMKLC_BF16_FP8HIDDEN */
  uint32_t optimizer;          /* PMKLC_ADAM or PMKLC_SGD */
  float lr;                    /* learning rate of the Backward Controller (§4.2.6) */
  float alpha_init;            /* initial mixing weight alpha of Eq. (1) */
  uint32_t smp_mode;           /* PMKLC_SMP_* (§4.3, Fig. 5) */
  float smp_fraction;          /* f: share of a parent's steps before it hands over (paper: 0.05) */
  uint32_t count_order;        /* order m of the count model, 0..7 */
  uint32_t fallback;           /* 0: network only; 1: per block, the count model when it is smaller
                                  (needs lanes_per_block <= 1024); 2: count model only */
  uint64_t seed;               /* seed of the dynamic model's initialisation */
  const float *static_weights; /* host FP32 static parameters (the MLP layout above, or with
                                  static_arch 1 or 2 the BiGRU layout of pmklc_predict_bigru);
                                  NULL if unused */
  uint32_t lane_tokens;        /* 0: a block of l tokens gets min(lanes_per_block, l) lanes; else
                                  min(lanes_per_block, l, ceil(l / lane_tokens)), so lanes of uneven
                                  blocks take about the same number of steps */
  uint32_t overlap_mask;       /* 1 (s < k; not in the paper): token j >= 1 of a lane is coded over
                                  the 4^s tokens that share their first k - s digits with the last
                                  k - s digits of token j - 1 (the only ones that can follow):
                                  uniform over them in the first t symbols, else the softmax of
                                  their mixed logits, trained on that slice's cross entropy */
  uint32_t update_path;        /* where the BF16 forms apply the optimiser to W1 and W2 (an
                                  implementation choice: every coded byte is the same either way):
                                  PMKLC_UPDATE_AUTO (0, by the size of the run), PMKLC_UPDATE_STREAM
                                  (1, gradients stored, then the streaming optimiser) or
                                  PMKLC_UPDATE_FUSED (2, in the epilogues of the gradient GEMMs on the
                                  tcgen05 engine, where that engine runs them; else as 1) */
  uint32_t private_model;      /* Model Selector (§4.2.1): 0 = the static model as given (or none);
                                  1 = a static private model (SPrM, §4.2.3) of the static shape
                                  (emb_s, ctx_s, hid_s), pre-trained on the input by the library's
                                  own kernels (as pmklc_train_model, starting from static_weights
                                  when use_static, else from the seeded init), stored in the
                                  container in BF16 and used in the static slot of Eq. (1); 2 =
                                  automatic: SPrM for inputs above 500 MB (5e8 bases), else as 0 */
  uint32_t private_epochs;     /* pre-training passes over the input (0 = 1) */
  uint64_t private_bases;      /* bases at the head of the input that pre-training reads (0 = all) */
  uint64_t private_threshold;  /* private_model 2 selects SPrM for inputs above this many bases
                                  (0 = 5e8, the paper's 500 MB; smaller values scale the rule down) */
  uint32_t gemm_tiles;         /* tile variant of the tcgen05 row GEMMs (hidden, logits, dh, dX):
                                  0 the default plan, 1 column tiles of at most 128, 2 at most 64;
                                  like update_path an implementation choice that leaves every coded
                                  byte unchanged (the reduction over K of each output element is the
                                  same); both are recorded in the container's variant field, so
                                  decompression runs the same kernels */
  uint32_t static_arch;        /* architecture of the static predictor: 0 the MLP of the layout above
                                  (emb_s, ctx_s, hid_s); 1 or 2 the BiGRU static predictor of
                                  pmklc_predict_bigru with that many BiGRU layers (§4.2.3 SPrM: one,
                                  §4.2.2 SPuM: two), E = emb_s, t = ctx_s, GRU width hid_s, weights
                                  in its layout (pmklc_bigru_count floats).  It needs use_static,
                                  private_model 0 and precision PMKLC_FP32_PLAIN or
                                  PMKLC_BF16_BATCHED; its Linear layer forms the static h (128
                                  wide) and its Dense layer runs on the MLP logits kernels */
} pmklc_model_cfg;

int pmklc_abi_version(void);
const char *pmklc_strerror(int rc);
void pmklc_free(void *p);

/* Number of FP32 parameters of an MLP predictor with alphabet 4^k (0 outside the accepted
 * widths: 1 <= k <= 8, 1 <= emb, ctx <= 4096, 1 <= hid <= 65535). */
size_t pmklc_model_count(uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid);

/*
 * Seeded initial parameters of an MLP predictor (the paper's "randomly
 * initialized parameters", §4.3; the paper names no generator: counter-based splitmix64 draws
 * scaled by 1 for the embedding and 1/sqrt(fan_in) for W1, W2; biases 0).
 * out: host array of pmklc_model_count(k, emb, ctx, hid) floats.
 */
int pmklc_init_model(uint32_t k, uint32_t emb, uint32_t ctx, uint32_t hid, uint64_t seed, float *out);

/*
 * Pre-training of a static predictor (paper §4, MSGD pre-training of the static
 * public model, Fig. 2(a)) with the library's own forward/backward/optimiser
 * kernels: the n training bases are tokenised with (cfg->s, cfg->k) and cut into
 * cfg->lanes_per_block lanes; the dynamic-model loop of pmklc_compress runs over
 * them `epochs` times without coding (each epoch continues from the previous
 * state).  The trained FP32 parameters of shape (emb_d, ctx_d, hid_d), starting
 * from pmklc_init_model(..., cfg->seed), go to out (host,
 * pmklc_model_count(k, emb_d, ctx_d, hid_d) floats).  cfg->use_static must be 0.
 * Without a static model the mixer of Eq. (1) forms the logits (1 - alpha) L, and alpha
 * trains alongside the weights; the returned logits layer (W2, b2) is multiplied by the final
 * (1 - alpha) (in FP32), so the returned predictor alone computes the logits the training fitted.
 */
int pmklc_train_model(const uint8_t *seq, size_t n, const pmklc_model_cfg *cfg, uint32_t epochs, void *stream,
                      float *out);

/*
 * Kernel-variant autotuner (measurement support; the paper has no counterpart): times a
 * compression of the heads of all n_blocks blocks (the first head_bases bases of each, so every
 * global step has the full run's groups and lanes) under each candidate variant code
 * (gemm_tiles | update_path << 2), picks the fastest and sets cfg->gemm_tiles and cfg->update_path.
 * Every variant gives the same container.  d_seq: the device input (n bases); ms (optional, host):
 * n_variants times in milliseconds.  Errors: EINVAL (bad cfg, codes, block lengths), ENOMEM, ECUDA.
 */
int pmklc_autotune_variant(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                           uint64_t head_bases, pmklc_model_cfg *cfg, const uint32_t *variants, size_t n_variants,
                           void *stream, float *ms);

/* Default configuration for (s,k) with dynamic model (E,t,H) = (emb, ctx, hid). */
void pmklc_default_cfg(pmklc_model_cfg *cfg, uint32_t s, uint32_t k, uint32_t emb, uint32_t ctx,
                       uint32_t hid);

/*
 * Compress n ASCII bases (A, C, G, T only) split into n_blocks blocks
 * (block_lens sums to n; the paper's Data Chunker, §4.3) into a container
 * (format: an 80-byte header, per-block records, then the lane payloads).  The static weights are not stored, only their
 * hash (§4.2.2: the public static model is part of the compressor).
 * Output: *out (library-allocated, pmklc_free) of *out_len bytes.
 * At most 32,767 blocks per call (each block is a model group, and both models' groups share
 * one grid dimension of the GEMM launches).
 * Errors: EINVAL (bad cfg, non-ACGT byte, block lengths, more than 32,767 blocks), ENOMEM, ECUDA.
 */
int pmklc_compress(const uint8_t *seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                   const pmklc_model_cfg *cfg, void *stream, uint8_t **out, size_t *out_len);

/*
 * Inverse of pmklc_compress (paper §2, decompression: the decoder replays
 * the same model updates).  static_weights/static_count must be the ones
 * used to compress when the container says a static model was used, unless it
 * stores its own static private model (then they are not used); static_count
 * is their number of floats (pmklc_model_count, or pmklc_bigru_count for a
 * BiGRU static predictor, flag bits 4-5 of the container).
 * Outputs: *seq (*n bases) and *block_lens (*n_blocks entries), both
 * library-allocated.  Errors: ECORRUPT, EMODEL, ENOMEM, ECUDA, ETIMEOUT.
 */
int pmklc_decompress(const uint8_t *in, size_t in_len, const float *static_weights, size_t static_count,
                     void *stream, uint8_t **seq, size_t *n, uint64_t **block_lens, size_t *n_blocks);

/*
 * Autotuner of the batch size (lanes per block; the paper's bs, §5.8): compresses
 * the first `sample_blocks` blocks of the device input once per candidate value
 * (after one untimed warm-up), timing each on `stream`, and picks the fastest
 * candidate whose coded size is at most (1 + max_rel_size) times the size
 * coded with candidates[0] (the reference).  cfg->lanes_per_block is set to the
 * choice; sizes (bytes) and times (ms) per candidate go to the optional arrays.
 * Errors as pmklc_compress_dev.
 */
int pmklc_autotune_lanes(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                         size_t sample_blocks, pmklc_model_cfg *cfg, const uint32_t *candidates,
                         size_t n_candidates, float max_rel_size, void *stream, uint64_t *sizes, float *ms);

/*
 * Upper bound of the container size of pmklc_compress_dev for this input (0 for an invalid
 * configuration or more than 32,767 blocks).  Per lane: at most 3 bytes per token + 8 for the network's stream (24-bit
 * totals); with fallback 2 (count model only) at most 2 bytes per base + 8 (count totals stay
 * below 2^13).  No input, however adversarial, makes a valid compression exceed it.
 */
size_t pmklc_compress_bound(size_t n, const uint64_t *block_lens, size_t n_blocks, const pmklc_model_cfg *cfg);

/*
 * Device-resident forms: input and output in device memory (the container
 * header is assembled on the host and copied in).  d_out must hold
 * pmklc_compress_bound() bytes; *out_len receives the container size.
 */
int pmklc_compress_dev(const uint8_t *d_seq, size_t n, const uint64_t *block_lens, size_t n_blocks,
                       const pmklc_model_cfg *cfg, void *stream, uint8_t *d_out, size_t out_cap,
                       size_t *out_len);
/* d_seq must hold seq_cap bytes; *n receives the number of bases. */
int pmklc_decompress_dev(const uint8_t *d_in, size_t in_len, const float *static_weights,
                         size_t static_count, void *stream, uint8_t *d_seq, size_t seq_cap, size_t *n);

/* ---------------------------------------------------------------------------
 * Single-step entry points (device buffers), each running exactly the device
 * code the compressor uses for that step.  They exist so each step can be
 * checked on its own against the oracle.
 */

/*
 * (s,k)-mer encoding, GskE (paper §4.1, Fig. 3): d_tokens[j] =
 * sum_m 4^(k-1-m) code(d_seq[j*s+m]) for j < l = floor((n-k)/s)+1 (0 if n < k);
 * the n - covered trailing bases go to d_tail as codes 0..3 (at most 7).
 * d_tokens holds l entries.  *n_tokens receives l.  EINVAL on a non-ACGT byte
 * or n > 2^56.
 */
int pmklc_tokenize(const uint8_t *d_seq, size_t n, uint32_t s, uint32_t k, uint16_t *d_tokens,
                   uint8_t *d_tail, size_t *n_tokens, void *stream);

/*
 * Quantisation of probabilities into an integer frequency table (paper §2
 * step 3; the paper does not say how P becomes integers): for each of `rows` rows of A probabilities,
 * freq_j = 1 + floor(P_j*(2^24 - A)) (FP32 product), the remainder added to
 * the first maximal entry.  d_P: rows x A FP32; d_freq: rows x A uint32.
 * rows <= 2^26 (one warp per row), else EINVAL.
 */
int pmklc_quantize(const float *d_P, size_t rows, uint32_t A, uint32_t *d_freq, void *stream);

/*
 * Probability Mixer, Eq. (1), + softmax + quantisation, per row:
 * P = softmax(alpha*Lu + (1-alpha)*Lm) (Lu ignored when use_static = 0).
 * d_Lu, d_Lm: rows x A FP32 logits; d_P: rows x A FP32; d_freq: rows x A.
 * rows <= 2^26, else EINVAL.
 */
int pmklc_mix_quantize(const float *d_Lu, const float *d_Lm, size_t rows, uint32_t A, float alpha,
                       uint32_t use_static, float *d_P, uint32_t *d_freq, void *stream);

/*
 * Range coding of independent streams (paper §2 step 3; the paper leaves its entropy encoder unspecified:
 * a byte-oriented range coder with a 56-bit window, carries through a cache byte).
 * Stream i codes L symbols d_sym[i*L + j] with frequency tables
 * d_freq[(i*L + j)*A .. +A) (each summing to 2^24).  Output bytes of stream i
 * go to d_out[i*cap ...], their count to d_len[i]; cap >= 3*L + 8 always
 * suffices.  ENOSPC if a stream overflows cap.  EINVAL if a symbol is >= A, or
 * the table entry it codes is 0 or its interval ends past 2^24 (that stream
 * stops there), or n_streams or L exceeds 2^31 - 1.
 */
int pmklc_range_encode(const uint32_t *d_freq, const uint16_t *d_sym, uint32_t n_streams, uint32_t L,
                       uint32_t A, uint8_t *d_out, uint32_t cap, uint32_t *d_len, void *stream);
/* Decoding of the streams written by pmklc_range_encode (same layout): stream i
 * reads at most min(d_len[i], cap) bytes (bytes past them read as 0).  EINVAL if
 * a table's entries end below the decoded target or run past 2^24 (that stream
 * stops there). */
int pmklc_range_decode(const uint32_t *d_freq, const uint8_t *d_in, const uint32_t *d_len, uint32_t n_streams,
                       uint32_t L, uint32_t A, uint32_t cap, uint16_t *d_sym, void *stream);

/*
 * Predictor forward (paper §2 step 3; MLP of the measured configurations):
 * logits[r] = relu(X_r W1 + b1) W2 + b2 with X_r the embeddings of the t
 * context tokens d_ctx[r*t .. r*t+t) (oldest first).  d_params in the model
 * layout for (A=4^k, E, t, H); d_logits rows x A.  precision as in the cfg.
 * Widths as in the cfg; rows <= 2^24 and rows x H < 2^31, else EINVAL.
 */
int pmklc_predict(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t H,
                  const uint16_t *d_ctx, size_t rows, uint32_t precision, float *d_logits, void *stream);

/*
 * BiGRU static predictor (paper §4.2.2: the static public model SPuM reads the
 * t context tokens through an embedding of width E (16 in the paper), two
 * bidirectional GRU layers and a Linear and a Dense layer of width 128; §4.2.3:
 * the static private model SPrM has the same structure with one BiGRU layer).
 * The paper gives the layers, not their equations; the reading used is the GRU
 * with the reset gate on the recurrent projection after its bias,
 *     r = sigmoid(Wi_r x + bi_r + Wh_r h + bh_r),  z = sigmoid(Wi_z x + bi_z + Wh_z h + bh_z),
 *     n = tanh(Wi_n x + bi_n + r (Wh_n h + bh_n)),  h' = (1 - z) n + z h,  h = 0 at the start,
 * a forward GRU over the positions oldest first and a backward one newest
 * first per layer (layer output [h^f_p, h^b_p], the next layer's input), the
 * summary u = [forward state after the newest token, backward state after the
 * oldest], q = relu(W3 u + b3) (128 wide) and logits L = q W4 + b4.
 * Parameters: one FP32 array
 *     Emb[A][E]
 *     for layer l = 0 .. layers-1, for direction forward then backward:
 *         Wi[3Hg][in_l] | Wh[3Hg][Hg] | bi[3Hg] | bh[3Hg]   (gate rows r, z, n;
 *                                                           in_0 = E, in_1 = 2Hg)
 *     W3[128][2Hg] | b3[128] | W4[128][A] | b4[A]
 * (row-major, A = 4^k; the size does not depend on t).  Hg is the GRU width per
 * direction, which the paper does not state.
 * pmklc_bigru_count: the number of parameters (0 for shapes outside those
 * built: E in {8, 16, 32}, Hg in {16, 32}, layers 1 or 2, 1 <= k <= 8).
 * pmklc_predict_bigru: for rows d_ctx[r*t .. r*t+t) (oldest first; 1 <= t <=
 * 4096, rows <= 2^24) writes q into d_q (rows x 128, optional) and the logits
 * into d_logits (rows x A, optional; at least one of the two).  FP32 on the CUDA
 * cores.  It allocates its scratch (t x 2Hg x rows floats with two layers) on
 * `stream`.  A token >= A is read as token 0 and the call returns EINVAL.
 */
size_t pmklc_bigru_count(uint32_t k, uint32_t E, uint32_t Hg, uint32_t layers);
int pmklc_predict_bigru(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t Hg, uint32_t layers,
                        const uint16_t *d_ctx, size_t rows, float *d_q, float *d_logits, void *stream);

/*
 * One update of G dynamic models from their own batches of M rows each
 * (paper §2 step 4, Eq. 1 and Eq. 2 with the Backward Controller):
 * forward of the dynamic (and, if use_static, static) predictor, Eq. (1)
 * mixing, softmax, mean cross entropy over the M rows, backward, and the
 * optimiser step at update count tau (1-based).
 *   d_params/d_m/d_v: G x P (P = pmklc_model_count of the dynamic shape),
 *     updated in place; d_alpha/d_alpha_m/d_alpha_v: G entries, in place.
 *   d_ctx: G*M rows of t_eff = max(ctx_d, use_static ? ctx_s : 0) tokens,
 *     oldest first; each model reads the last t of its own context length.
 *   d_target: G*M tokens.  d_static: the static parameters (if use_static).
 *   d_P (optional, G*M x A) receives the mixed probabilities before the
 *   update; d_grad (optional, G x P) the gradient; d_dalpha (optional, G).
 * 1 <= G <= 32,767 (the limit of pmklc_compress's blocks), else EINVAL.
 * The static model here is an MLP: cfg->static_arch other than 0 is EINVAL.
 */
int pmklc_train_step(const pmklc_model_cfg *cfg, uint32_t G, uint32_t M, float *d_params, float *d_m,
                     float *d_v, float *d_alpha, float *d_alpha_m, float *d_alpha_v, const float *d_static,
                     const uint16_t *d_ctx, const uint16_t *d_target, uint32_t tau, float *d_P, float *d_grad,
                     float *d_dalpha, void *stream);

/*
 * FP8 (E4M3) form of a frozen static predictor (the paper's static public model
 * is frozen, §4.2.2 and Fig. 2(a); its precision is not stated): one scale per
 * channel, s = amax / 448 (1 for an all-zero channel), code = E4M3(w / s)
 * rounded to nearest even and saturated at 448, both divisions in FP32.
 * Channels: the whole embedding table; each hidden unit (a row of W1t); each
 * logit (a column of W2).  The compressor applies this to the static weights
 * when cfg->precision is PMKLC_BF16_FP8STATIC (PMKLC_BF16_FP8HIDDEN uses the
 * embedding and W1 codes only); the entry point exposes it.
 *   d_params: device FP32 parameters (layout above) of shape (k, E, t, H);
 *     E must be a multiple of 16 for the FP8 forward (not checked here).
 *   d_codes: device, 4^k*E + H*t*E + 4^k*H bytes: Emb codes [A][E], W1t codes
 *     [H][t*E], W2 codes transposed [A][H].
 *   d_scales: device, 1 + H + 4^k floats: s_emb, s_w1[H], s_w2[A].
 * Errors: EINVAL (shape, NULL pointers), ECUDA.
 */
int pmklc_quantize_static_fp8(const float *d_params, uint32_t k, uint32_t E, uint32_t t, uint32_t H,
                              uint8_t *d_codes, float *d_scales, void *stream);

/*
 * Failure-detection self-test (the paper has no counterpart: a library service).
 * Every wait of the library's kernels is bounded: on expiry the kernel sets an
 * error bit, lets its copies land, frees its tensor memory and returns, and the
 * call returns PMKLC_ETIMEOUT with the CUDA context intact.  This runs that path
 * on its own: one thread polls, at most `polls` times, an mbarrier that expects
 * an arrival which never comes.  Returns PMKLC_ETIMEOUT (the expected outcome),
 * EINVAL for polls = 0 or above 2^30, ECUDA on a CUDA error.
 */
int pmklc_wait_selftest(uint64_t polls, void *stream);

/* CRC-32 (IEEE 802.3, reflected, as zlib) of n device bytes. */
int pmklc_crc32(const uint8_t *d_data, size_t n, uint32_t *crc, void *stream);

/*
 * The same CRC-32 computed without allocating any device memory (the paper has
 * no counterpart: this is a library service).  For callers that cannot call
 * cudaMalloc: processes whose device memory is handed out entirely by another
 * framework's pool allocator, and latency-sensitive loops that must not pay for
 * an allocation.  Its scratch is a fixed array in the library's device memory
 * (about 256 KiB, kept on every device that loads the library until the
 * process exits), so n is limited to 256 MiB plus up to 4110 bytes of unaligned
 * head and ragged tail; larger inputs return PMKLC_EINVAL before touching any
 * memory.  The first call on a device looks up the array's device address once
 * (with that device current); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents; nothing in it
 * must start at zero, but calls that overlap on the GPU (other streams or host
 * threads) race on it and must be serialised by the caller.
 */
int pmklc_crc32_noalloc(const uint8_t *d_data, size_t n, uint32_t *crc, void *stream);

/* Last run's statistics (per thread): compressed payload split and timings.  After a
 * compression, net_bytes and count_bytes are what the network's and the count model's codings of
 * every block cost (lane payloads and their length fields, as the judge compares them; 0 for a
 * coding that did not run: the count model with fallback 0, the network with fallback 2). */
typedef struct {
  uint64_t net_blocks, count_blocks;
  uint64_t global_steps;
  uint64_t kernel_launches;
  double ms_total;
  uint64_t net_bytes, count_bytes;
} pmklc_stats;
int pmklc_last_stats(pmklc_stats *st);

/*
 * Measurement support (not part of the paper's method): sampled per-kernel
 * timing.  pmklc_profile_enable(every) brackets every kernel launch of every
 * `every`-th global step (0 = off) with CUDA events on the launching stream,
 * together with the launch's algorithmic work (FLOPs of its contraction or
 * bytes it must move).  pmklc_profile_read() waits for the events, returns up
 * to `max` per-kernel totals (*n = number of kernels seen) and clears them.
 */
typedef struct {
  char name[32];
  uint64_t launches;
  double ms, flops, bytes;
} pmklc_kernel_prof;
int pmklc_profile_enable(int every);
int pmklc_profile_read(pmklc_kernel_prof *out, int max, int *n);

#ifdef __cplusplus
}
#endif
#endif /* PMKLC_H */
