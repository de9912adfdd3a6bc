// Declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ptycho {

// MODE_GRAD stores every slice's entering wave and exit-wave gradient.
// Recompute mode (checkpoint every ckpt_L slices, K segments) is K launches:
// MODE_GRAD_RC runs the forward model keeping the checkpoints and the last
// segment's waves, the residual, and the adjoint through the last segment;
// MODE_RC_SEG (segment ChainArgs::seg = K-2 .. 0) rebuilds one segment's
// waves from its checkpoint and runs the adjoint through it.  Both write the
// segment's finished gradient patches conj(psi_s) g_phi_s over its waves.
enum ChainMode { MODE_FORWARD = 0, MODE_LOSS = 1, MODE_GRAD = 2, MODE_GRAD_RC = 3, MODE_RC_SEG = 4 };

// Arguments of the per-position slice-chain kernel.  Positions
// [pos_begin, pos_begin + n_pos) of the call are processed, one per block.
struct ChainArgs {
  const int2* pos;        // [N] (y, x)
  int pos_begin;
  int n_pos;
  const float2* probe;    // [M][M]
  const float2* obj;      // [S][H][W]
  const float2* obj_dir;  // [S][H][W] or null: evaluate at obj + obj_step * obj_dir
  const float2* probe_dir;// [M][M] or null: evaluate at probe + probe_step * probe_dir
  float obj_step, probe_step;
  const float* meas;      // [N][M][M] FFT order
  int S, H, W;
  const float2* tw;       // [M]   w_M^e = exp(-2 pi i e / M)
  const float2* hs;       // [M]   one separable factor of the propagator, times 1/M
  const float2* h2;       // [M][M] the propagator h(ky) h(kx) / M^2 (register-resident kernels)
  int ws_n;               // positions the workspace holds (slice stride of ws_psi / ws_gphi)
  int ckpt_L;             // recompute mode: checkpoint every ckpt_L slices
  int seg;                // MODE_RC_SEG: the segment differentiated by this launch
  float2* ws_psi;         // GRAD: [S-1][ws_n][M][M] waves entering slices 1..S-1
                          // recompute: [K-2 checkpoints | ckpt_L segment waves, then
                          // patches | 1 parked adjoint state][ws_n][M][M]
  float2* ws_gphi;        // GRAD: [S][ws_n][M][M] gradient w.r.t. each slice's exit wave
  float2* ws_gp;          // [ws_n][M][M]      per-position probe gradient
  double* loss_part;      // [n_pos]
  float2* psi_out;        // [N][M][M] or null (forward mode)
  float* int_out;         // [N][M][M] or null (forward mode)
  int* status;            // device error word (PTYCHO_ERR_POSITION on a bad window)
  int selftest_timeout;   // PTYCHO_FLAG_SELFTEST_TIMEOUT: the split-product kernel issues no MMAs
};

// Gradient-mode chains of several problems (same window M = 64 or 128, FP32,
// every wave kept) in one launch: a[p] is problem p's ChainArgs for its
// current chunk, whose blocks are [start[p], start[p + 1]).  Passed by value
// as the kernel's parameter (kMultiChainMax entries keep it under 4 KB).
constexpr int kMultiChainMax = 16;
struct MultiChainArgs {
  int n;
  int start[kMultiChainMax + 1];
  ChainArgs a[kMultiChainMax];
};
static_assert(sizeof(MultiChainArgs) <= 4096, "kernel parameters of the multi-problem chain exceed 4 KB");

// chain_kernels.cu
cudaError_t launch_chain_multi(int M, const MultiChainArgs& m, cudaStream_t st);
int chain_threads(int M);
int chain_blocks_per_sm(int M);  // resident gradient-mode blocks per SM (0 if unknown)
size_t chain_smem_bytes(int M);
cudaError_t chain_prepare(int M);  // raise the dynamic shared-memory limit
cudaError_t launch_chain(int M, ChainMode mode, const ChainArgs& a, cudaStream_t st);

// chain_tc.cu (BF16 or F16 hi/lo split DFT products on tcgen05, M = 128)
size_t chain_tc_smem_bytes();
cudaError_t chain_tc_prepare();
cudaError_t launch_chain_tc(ChainMode mode, const ChainArgs& a, const uint32_t* cplanes, bool f16,
                            cudaStream_t st);

// chain_gm.cu (any window M = 2^a 3^b, 8 <= M <= 4096, FP32)
struct GmPlan {
  int n;      // radix stages
  int r[16];  // radices (4, 2, 3)
};
bool gm_supported(int M, GmPlan* plan);
size_t gm_fft_smem_bytes(int M);
cudaError_t gm_prepare(int M);
cudaError_t launch_chain_gm(ChainMode mode, const ChainArgs& a, float2* wv, int M, int* n_launches,
                            cudaStream_t st);

// reduce_kernels.cu
constexpr int kDefaultTile = 32;  // default owner tile of the object-gradient accumulation
struct AccumArgs {
  const int2* pos;
  int pos_begin, n_pos;
  int M, S, H, W;
  int tile_h, tile_w;
  const float2* probe;      // wave entering slice 0 (= probe)
  int ws_n;                 // slice stride (positions) of ws_psi / ws_gphi
  const float2* ws_psi;     // [S-1][ws_n][M][M]
  const float2* ws_gphi;    // [S][ws_n][M][M]
  float2* grad_obj;         // [S][H][W]
  int accumulate;           // 0: overwrite the slices' gradient, 1: add
  int patch_mode;           // 1: ws_gphi holds finished patches (ws_psi unused)
  int s_begin, n_slices;    // slices [s_begin, s_begin + n_slices) (n_slices 0: all S)
  int seg_slots;            // 1: slice s's arrays sit at slot s - s_begin of ws_psi /
                            // ws_gphi (a recompute segment); 0: ws_psi slot s - 1,
                            // ws_gphi slot s (every wave kept)
};
cudaError_t launch_accum_obj_grad(const AccumArgs& a, cudaStream_t st);
cudaError_t launch_probe_grad(const float2* ws_gp, int n_pos, int M, float2* part, int n_split,
                              float2* grad_probe, int accumulate, cudaStream_t st);
cudaError_t launch_loss_accum(const double* loss_part, int n, double* acc, int accumulate,
                              cudaStream_t st);
cudaError_t launch_axpy(float2* y, const float2* x, const float2* base, double alpha, size_t n,
                        cudaStream_t st);  // y = base + alpha * x
cudaError_t launch_norm2(const float2* x, size_t n, double* part, int n_part, double* out,
                         int slot, cudaStream_t st);
cudaError_t launch_potential_to_transmission(const float* V, float2* O, double sigma, size_t n, cudaStream_t st);
cudaError_t launch_potential_grad(const float2* O, const float2* g, float* gV, double sigma, size_t n,
                                  cudaStream_t st);
cudaError_t launch_check_positions(const int2* pos, int n, int M, int H, int W, int* status,
                                   cudaStream_t st);

}  // namespace ptycho
