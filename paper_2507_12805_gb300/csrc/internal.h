// Host-side interfaces between the translation units of libpmklc.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace pmklc {

// profile.cu ----------------------------------------------------------------
// Work of the current global step, set by the step loop before its launches.
struct StepWork {
  double pred_rows;     // predicted (and trained) lane rows over all groups
  double train_groups;  // groups that update their model
};
void prof_step(int T, const StepWork &w);
void prof_stop_sampling();
// True while sampled profiling is on: the step loop then runs every kernel on the caller's stream,
// so each sampled kernel's event time is its own duration (no concurrent kernels share its SMs).
bool prof_enabled();
const StepWork &prof_work();
// Brackets one kernel launch with events when the current step is sampled.
class ProfScope {
 public:
  ProfScope(const char *name, double flops, double bytes, cudaStream_t st);
  ~ProfScope();

 private:
  const char *name_;
  double flops_, bytes_;
  cudaStream_t st_;
  bool active_;
  void *a_ = nullptr;
};

// Raises `func`'s dynamic shared-memory limit to at least `bytes` on the current device: one
// attribute call per (kernel, device, larger size), under a process-wide mutex, so host threads
// driving several devices share it safely.  False when the attribute call failed (the error stays
// recorded for the caller's cudaGetLastError).
bool smem_optin(const void *func, int bytes);

// tokenize.cu ---------------------------------------------------------------
// Validation (kErrBadBase in *d_err for a byte other than A, C, G, T) and tokens of every block:
// block b has bases [base_off[b], base_off[b+1]) of d_seq (n bytes) and tokens [tok_off[b],
// tok_off[b+1]) in d_tokens.  d_cta is tokenize_ctas(base_off) on the device: the first CTA of
// every block (n_blocks + 1 entries, the last one n_cta), then the block of every CTA (n_cta entries).
std::vector<int> tokenize_ctas(const std::vector<long long> &base_off);
void launch_validate_tokenize(const uint8_t *d_seq, size_t n, const long long *d_base_off, const long long *d_tok_off,
                              const int *d_cta, int n_blocks, int n_cta, int s, int k, uint16_t *d_tokens,
                              int *d_err, cudaStream_t st);
// Tail codes of every block (at most 7 per block) into d_tail[b*8 + i].
void launch_tails(const uint8_t *d_seq, const long long *d_base_off, const long long *d_tok_off, int n_blocks,
                  int s, int k, uint8_t *d_tail, cudaStream_t st);
// Inverse of tokenize for the blocks with d_sel[b] != 0: writes ASCII bases; sets kErrCorrupt
// when overlapping windows disagree.
void launch_detokenize(const uint16_t *d_tokens, const uint8_t *d_tail, const long long *d_base_off,
                       const long long *d_tok_off, const int *d_sel, int n_blocks, long long n_bases, int s, int k,
                       uint8_t *d_seq, int *d_err, cudaStream_t st);
int crc32_device(const uint8_t *d_data, size_t n, uint32_t *crc, cudaStream_t st);

// fp8static.cu ---------------------------------------------------------------
// FP8 (E4M3) form of a frozen model of shape d: codes [Emb A x E][W1t H x tE][W2 transposed A x H]
// (fp8_code_bytes) and scales [s_emb][s_w1: H][s_w2: A] (fp8_scale_count).
size_t fp8_code_bytes(const Dims &d);
size_t fp8_scale_count(const Dims &d);
void launch_quantize_fp8(const float *d_params, const Dims &d, uint8_t *d_codes, float *d_scales, cudaStream_t st);
// c1[h] = s_emb * s_w1[h], the hidden layer's combined scale
void launch_fp8_hidden_scale(const float *d_scales, const Dims &d, float *d_c1, cudaStream_t st);

// bigru.cu -------------------------------------------------------------------
// The BiGRU static predictor (§4.2.2 SPuM with two layers, §4.2.3 SPrM with one): element offsets
// of its flat FP32 parameters, Emb [A][E], then per layer l and direction d (forward, backward)
// Wi [3 Hg][in_l] | Wh [3 Hg][Hg] | bi [3 Hg] | bh [3 Hg] (gate rows r, z, n; in_0 = E, in_1 = 2 Hg),
// then W3 [kGruDense][2 Hg] | b3 [kGruDense] | W4 [kGruDense][A] | b4 [A].
constexpr int kGruDense = 128;  // width of the Linear layer (§4.2.2)
struct GruOff {
  size_t emb, wi[2][2], wh[2][2], bi[2][2], bh[2][2], w3, b3, w4, b4, count;
};
GruOff gru_offsets(int A, int E, int Hg, int layers);
// the shapes the kernel is built for: E in {8, 16, 32}, Hg in {16, 32}, 1 or 2 layers, 1 <= t <= 4096
bool gru_shape_ok(int k, int E, int t, int Hg, int layers);
int gru_smem_bytes(int Hg);
// The static h of the lanes predicted at global step T (p.hs in the FP32 form, p.hs_b in the BF16
// forms), formed by the BiGRU static predictor of p.st_gru.
void launch_bigru_static(const Plan &p, int T, cudaStream_t st);

// countmodel.cu --------------------------------------------------------------
void launch_count_step(const Plan &p, const CountPlan &c, int T, cudaStream_t st);
void launch_count_init(const Plan &p, const CountPlan &c, int encode, cudaStream_t st);
void launch_count_finish(const Plan &p, const CountPlan &c, uint32_t *d_lane_len, cudaStream_t st);

// mixcode.cu -----------------------------------------------------------------
void launch_mixcode(const Plan &p, int T, cudaStream_t st);
void launch_coder_init(const Plan &p, int encode, cudaStream_t st);
void launch_coder_finish(const Plan &p, uint32_t *d_lane_len, cudaStream_t st);

// predictor.cu ---------------------------------------------------------------
void launch_forward(const Plan &p, int T, cudaStream_t st);
void launch_backward(const Plan &p, int T, cudaStream_t st);
void launch_update(const Plan &p, int T, cudaStream_t st);
void launch_backward_update(const Plan &p, int T, cudaStream_t st);
// gradient of every group (embedding part from the fixed-point accumulators) into d_out (G x P)
void launch_export_grad(const Plan &p, float *d_out, cudaStream_t st);
// Auxiliary streams of a run's step loop: independent kernels of a step are forked onto them and
// joined back by events (fork/join events reused every step).
struct StepStreams {
  cudaStream_t aux[3];  // 0: count model, dW2; 1: dX; 2: the static model's forward
  cudaEvent_t fork, join[2], count_done, mix_done, static_done;
};

// predictor_tc.cu: the BF16 form's GEMMs on tcgen05, for shapes with E % 8 == 0, H % 16 == 0,
// 4^k % 8 == 0 and a parameter count divisible by 8 (16-byte aligned per-group BF16 copies)
bool tc_supported(const Plan &p);
// which: kFwdDynamic and/or kFwdStatic (the static model's forward depends on the tokens only, so a
// step loop may run it on another stream)
constexpr int kFwdDynamic = 1, kFwdStatic = 2, kFwdBoth = 3;
void launch_forward_tc(const Plan &p, int T, cudaStream_t st, int which = kFwdBoth);
// partial embedding-gradient tables per group of the dX GEMM when it sums its tiles in FP32 by
// owner warps (small tables), else 0; *ct = its column tiles
int dx_partials(const Plan &p, int *ct);
// true when the dX GEMM stores its rows (Plan::dx_rows, NL x t*E FP32) for a separate sum into the
// embedding gradient: tables too large for the shared-memory forms
bool dx_rows_rule(const Plan &p);
// ... and then the number of bins (ranges of table rows) its pairs are listed by (Plan::emb_bin_off
// holds G x (bins + 1) offsets), else 0
int dx_rows_bins(const Plan &p);
// slice.cu: with overlap-masked coding (slice width 4^s of 16 to 64 tokens) the logits layer and dh
// formed over each row's coded slice only, reading every group's W2 about once per step.
// launch_slice_logits: problems zb .. zb + Z - 1 (z < G dynamic, z >= G static on group z - G)
bool slice_rule(const Plan &p);
void launch_slice_logits(const Plan &p, int T, cudaStream_t st, int zb, int Z);
void launch_slice_dh(const Plan &p, int T, cudaStream_t st);
// ss (optional): run dW2, dX and dW1 concurrently on st and ss->aux
void launch_backward_tc(const Plan &p, int T, cudaStream_t st, const StepStreams *ss);
// predictor_bf16.cu: the BF16 form (tcgen05 engine where tc_supported, else mma.sync)
void launch_forward_bf16(const Plan &p, int T, cudaStream_t st, int which = kFwdBoth);
// gradient GEMMs into the gradient buffer (the optimiser is launch_update)
void launch_backward_bf16(const Plan &p, int T, cudaStream_t st, const StepStreams *ss = nullptr);
void launch_to_bf16(const float *src, void *dst, size_t n, cudaStream_t st);
void launch_smp_copy(const Plan &p, const int *d_pairs, int n_pairs, cudaStream_t st);
void launch_init_groups(const Plan &p, const float *d_init, float alpha0, cudaStream_t st);

}  // namespace pmklc
