// Per-position multislice chain: forward model G (Sec. II-B), amplitude
// residual of Eq. 1 and the exact adjoint back to the slices and the probe
// (the per-position term of Eq. 2, Sec. III).
//
// One thread block owns one probe position for its whole slice chain; the
// wave never leaves the SM between slices.  Per slice s the forward pass
// multiplies by the object window O_s[y_i:y_i+M, x_i:x_i+M] (read straight
// from global memory, L2-resident) and, if s < S-1, propagates by
// FFT -> x h -> IFFT.  The exit wave is transformed to the detector; the
// residual gives the loss term and the seed of the adjoint, which runs the
// chain backwards with conjugated factors.
//
// Gradient mode writes, per position, the wave entering every slice s >= 1
// and the gradient w.r.t. every slice's exit wave (streaming stores); the
// object gradient conj(psi_s) * g_phi_s is formed and summed per object tile
// by the deterministic owner-computes reduction in reduce_kernels.cu.
//
// Recompute mode (checkpoint every L slices, K = ceil(S / L) segments) runs
// as K launches so that the workspace does not hold a patch per slice: the
// first (MODE_GRAD_RC) runs the forward model keeping only the checkpoints
// entering segments 1..K-2 and the waves of the last segment, then the
// residual and the adjoint through the last segment, writing its finished
// gradient patches conj(psi_s) g_phi_s over those waves and parking the
// adjoint state.  Each later launch (MODE_RC_SEG, segment j = K-2 .. 0)
// rebuilds segment j's waves from its checkpoint (or the probe) with the
// forward model's exact operations, runs the adjoint through the segment from
// the parked state and parks the state again (segment 0: the probe gradient).
// The host accumulates each segment's patches into the object gradient
// before the next launch overwrites them.
#include "fft2d.cuh"
#include "internal.h"
#include "../../include/ptycho.h"

namespace ptycho {

namespace {

// Elementwise over the pass-0 grouping (natural order), element (py, px).
template <class C, class F>
__device__ __forceinline__ void for_p0(int t, F&& f) {
  using P = PassShape<C, 0>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py0, px0;
    C::template base<0>(t, q, py0, px0);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        f(q * P::G + a * P::RX + b, py0 + a * P::SY, px0 + b * P::SX);
      });
    });
  });
}

// Elementwise over the pass-2 grouping (spectrum), frequency (ky, kx).
template <class C, class F>
__device__ __forceinline__ void for_p2(int t, F&& f) {
  using P = PassShape<C, 2>;
  t = opaque(t);
  static_for<0, P::Q>([&](auto qq) {
    constexpr int q = decltype(qq)::value;
    int py, px;
    C::template base<2>(t, q, py, px);
    const int ky0 = freq_y<C>(py), kx0 = freq_x<C>(px);
    static_for<0, P::RY>([&](auto aa) {
      constexpr int a = decltype(aa)::value;
      static_for<0, P::RX>([&](auto bb) {
        constexpr int b = decltype(bb)::value;
        f(q * P::G + a * P::RX + b, ky0 + C::ry(0) * C::ry(1) * a, kx0 + C::rx(0) * C::rx(1) * b);
      });
    });
  });
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

// The forward model's propagations multiply by the full propagator table
// (one rounding per element fewer; the residual amplifies the forward
// model's rounding), the adjoint's by the separable factors in shared memory.
#ifndef PTYCHO_PROP_TABLE
#define PTYCHO_PROP_TABLE 1
#endif
template <class C>
__device__ __forceinline__ void mul_prop_fwd(float2 (&v)[C::V], const float2* hs, const float2* h2, int t) {
#if PTYCHO_PROP_TABLE
  mul_table<C, false>(v, h2, t);
#else
  mul_separable<C, false>(v, hs, t);
#endif
}

// Recompute mode's finished patches are read once by the accumulation that
// follows each launch: streaming stores by default; plain stores (to keep a
// chunk's patches in L2 when the chunk is small enough) with
// PTYCHO_PATCH_STORE_CS=0.
#ifndef PTYCHO_PATCH_STORE_CS
#define PTYCHO_PATCH_STORE_CS 1
#endif
__device__ __forceinline__ void store_patch(float2* p, float2 v) {
#if PTYCHO_PATCH_STORE_CS
  __stcs(p, v);
#else
  *p = v;
#endif
}

}  // namespace


template <int M, int MODE>
__global__ void __launch_bounds__(Cfg<M>::T, Cfg<M>::MIN_BLOCKS) k_chain(const ChainArgs a) {
  const int il = blockIdx.x;
#include "chain_body.inc"
}

// Several problems' chunks in one launch (the batched workload): block b runs
// position b - start[p] of problem p's chunk, start[p] <= b < start[p + 1].
template <int M>
__global__ void __launch_bounds__(Cfg<M>::T, Cfg<M>::MIN_BLOCKS)
    k_chain_multi(const __grid_constant__ MultiChainArgs m) {
  constexpr int MODE = MODE_GRAD;
  __shared__ ChainArgs sa;
  const int b = blockIdx.x;
  int p = 0;
  while (p + 1 < m.n && b >= m.start[p + 1]) ++p;
  if (threadIdx.x == 0) sa = m.a[p];
  __syncthreads();
  const ChainArgs& a = sa;
  const int il = b - m.start[p];
#include "chain_body.inc"
}

int chain_threads(int M) { return M == 128 ? Cfg<128>::T : Cfg<64>::T; }

size_t chain_smem_bytes(int M) {
  return (size_t)M * M * sizeof(float2) + 2 * (size_t)M * sizeof(float2) +
         (size_t)(chain_threads(M) / 32) * sizeof(double);
}

template <int M>
static cudaError_t prepare_m() {
  const int bytes = (int)chain_smem_bytes(M);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_FORWARD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_GRAD_RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain<M, MODE_RC_SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chain_multi<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_chain<M, MODE_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t chain_prepare(int M) { return M == 128 ? prepare_m<128>() : prepare_m<64>(); }

int chain_blocks_per_sm(int M) {
  int n = 0;
  const cudaError_t e =
      M == 128 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<128, MODE_GRAD>, Cfg<128>::T,
                                                               chain_smem_bytes(128))
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_chain<64, MODE_GRAD>, Cfg<64>::T,
                                                               chain_smem_bytes(64));
  return e == cudaSuccess ? n : 0;
}

template <int M>
static cudaError_t launch_m(ChainMode mode, const ChainArgs& a, cudaStream_t st) {
  const dim3 grid(a.n_pos), block(Cfg<M>::T);
  const size_t smem = chain_smem_bytes(M);
  switch (mode) {
    case MODE_FORWARD: k_chain<M, MODE_FORWARD><<<grid, block, smem, st>>>(a); break;
    case MODE_LOSS: k_chain<M, MODE_LOSS><<<grid, block, smem, st>>>(a); break;
    case MODE_GRAD_RC: k_chain<M, MODE_GRAD_RC><<<grid, block, smem, st>>>(a); break;
    case MODE_RC_SEG: k_chain<M, MODE_RC_SEG><<<grid, block, smem, st>>>(a); break;
    default: k_chain<M, MODE_GRAD><<<grid, block, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_chain(int M, ChainMode mode, const ChainArgs& a, cudaStream_t st) {
  if (a.n_pos <= 0) return cudaSuccess;
  return M == 128 ? launch_m<128>(mode, a, st) : launch_m<64>(mode, a, st);
}

cudaError_t launch_chain_multi(int M, const MultiChainArgs& m, cudaStream_t st) {
  if (m.n < 0 || m.n > kMultiChainMax) return cudaErrorInvalidValue;
  if (m.n == 0 || m.start[m.n] <= 0) return cudaSuccess;
  const dim3 grid(m.start[m.n]), block(chain_threads(M));
  const size_t smem = chain_smem_bytes(M);
  if (M == 128)
    k_chain_multi<128><<<grid, block, smem, st>>>(m);
  else
    k_chain_multi<64><<<grid, block, smem, st>>>(m);
  return cudaGetLastError();
}

}  // namespace ptycho
