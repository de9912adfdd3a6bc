// ptycho_loss_grad_noalloc: the loss-and-gradient evaluation without any
// device allocation, for callers that cannot call cudaMalloc -- for example
// code running inside a custom device allocator or a memory-pool callback,
// or a host whose allocations are frozen after start-up (a pre-sized serving
// process).  The paper has no counterpart; it is a packaging of the same
// kernels.
//
// All scratch (tables, per-position waves, partial sums, the status word)
// lives in one file-scope device array of kScratchBytes that every GPU which
// loads the library holds until the process exits.  Positions are processed
// in chunks that fit in it, so any N works; a problem whose single position
// needs more than the array holds is rejected.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/ptycho.h"
#include "internal.h"

using namespace ptycho;

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kSplit = 4;                           // probe-gradient partials
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// The entry point reports through its return code only (it must not touch
// the library's heap-backed error text).  The message is kept for debuggers.
thread_local char g_msg[256];

int noalloc_fail(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  return code;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

bool device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" PTYCHO_API int ptycho_loss_grad_noalloc(const ptycho_params* params, const int32_t* pos_yx,
                                                   const ptycho_c64* probe, const ptycho_c64* obj,
                                                   const float* meas_I, double* loss_out,
                                                   ptycho_c64* grad_obj, ptycho_c64* grad_probe,
                                                   void* stream) {
  g_msg[0] = 0;
  if (!params) return noalloc_fail(PTYCHO_ERR_ARG, "params is NULL");
  const ptycho_params& p = *params;
  if (p.M != 64 && p.M != 128) return noalloc_fail(PTYCHO_ERR_UNSUPPORTED, "probe window M must be 64 or 128");
  if (p.S < 1 || p.H < p.M || p.W < p.M || p.N < 0 || p.precision != PTYCHO_FP32 || !(p.pixel_A > 0) ||
      !std::isfinite(p.lambda_A) || !std::isfinite(p.dz_A))
    return noalloc_fail(PTYCHO_ERR_ARG, "bad problem parameters");
  const int th = p.tile_h ? p.tile_h : kDefaultTile, tw_ = p.tile_w ? p.tile_w : kDefaultTile;
  if (th < 1 || tw_ < 1 || th * tw_ > 8192) return noalloc_fail(PTYCHO_ERR_ARG, "tile_h * tile_w must be in [1, 8192]");
  if (!loss_out) return noalloc_fail(PTYCHO_ERR_ARG, "loss_out is NULL");
  if (!device_ptr(probe) || !device_ptr(obj) || (p.N > 0 && (!device_ptr(meas_I) || !device_ptr(pos_yx))) ||
      (grad_obj && !device_ptr(grad_obj)) || (grad_probe && !device_ptr(grad_probe)))
    return noalloc_fail(PTYCHO_ERR_ARG, "arrays must be device pointers");
  // The kernels move positions and complex values as 8-byte int2 / float2
  // and intensities as floats: a misaligned array is an argument error here,
  // never a misaligned access on the device.
  if (!aligned8(probe) || !aligned8(obj) || (p.N > 0 && (!aligned8(pos_yx) || !aligned8(meas_I))) ||
      !aligned8(grad_obj) || !aligned8(grad_probe) || !aligned8(loss_out))
    return noalloc_fail(PTYCHO_ERR_ARG, "arrays must be 8-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;

  // Set-up, once per device with that device current: the device address of
  // the scratch array (its host-side name is only a stand-in) and the kernels'
  // shared-memory limit.
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(PTYCHO_ERR_CUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      if ((e = cudaGetSymbolAddress(&ptr, g_scratch)) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return noalloc_fail(PTYCHO_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      if ((e = chain_prepare(64)) != cudaSuccess || (e = chain_prepare(128)) != cudaSuccess)
        return noalloc_fail(PTYCHO_ERR_CUDA, "cudaFuncSetAttribute failed");
      g_scratch_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }

  // Carve the scratch: fixed part, then the per-chunk workspace.
  const int M = p.M;
  const size_t MM = (size_t)M * M;
  size_t off = 0;
  float2* d_tw = reinterpret_cast<float2*>(base + off); off = align_up(off + M * sizeof(float2));
  float2* d_hs = reinterpret_cast<float2*>(base + off); off = align_up(off + M * sizeof(float2));
  float2* d_h2 = reinterpret_cast<float2*>(base + off); off = align_up(off + MM * sizeof(float2));
  int* d_status = reinterpret_cast<int*>(base + off);   off = align_up(off + sizeof(int));
  double* d_loss = reinterpret_cast<double*>(base + off); off = align_up(off + sizeof(double));
  float2* gp_part = reinterpret_cast<float2*>(base + off); off = align_up(off + kSplit * MM * sizeof(float2));
  const size_t per_pos = (size_t)(2 * p.S - 1) * MM * sizeof(float2) + MM * sizeof(float2) + sizeof(double);
  if (off + per_pos + 4 * 256 > kScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "one position needs %zu bytes of scratch (M=%d, S=%d); the static scratch holds %zu", per_pos, M, p.S,
             kScratchBytes - off);
    return noalloc_fail(PTYCHO_ERR_UNSUPPORTED, buf);
  }
  const int chunk = (int)((kScratchBytes - off - 4 * 256) / per_pos);
  double* loss_part = reinterpret_cast<double*>(base + off); off = align_up(off + chunk * sizeof(double));
  float2* ws_gp = reinterpret_cast<float2*>(base + off);      off = align_up(off + chunk * MM * sizeof(float2));
  float2* ws_gphi = reinterpret_cast<float2*>(base + off);    off = align_up(off + (size_t)chunk * p.S * MM * sizeof(float2));
  float2* ws_psi = reinterpret_cast<float2*>(base + off);

  // Tables in FP64 on the host stack, rounded once to FP32.
  float2 tw[128], hs[128];
  const double two_pi = 6.283185307179586476925287;
  for (int k = 0; k < M; ++k) {
    const double ang = -two_pi * (double)k / (double)M;
    tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    const double f = (double)(k <= (M - 1) / 2 ? k : k - M) / ((double)M * p.pixel_A);
    const double ph = -M_PI * p.lambda_A * p.dz_A * f * f;
    hs[k] = make_float2((float)(std::cos(ph) / M), (float)(std::sin(ph) / M));
  }
  // The full propagator h(ky) h(kx) / M^2, staged through the stack 16 rows
  // at a time (a copy from pageable memory returns once its source is staged).
  for (int k0 = 0; k0 < M; k0 += 16) {
    float2 rows[16 * 128];
    for (int ky = k0; ky < k0 + 16; ++ky)
      for (int kx = 0; kx < M; ++kx) {
        const double fy = (double)(ky <= (M - 1) / 2 ? ky : ky - M) / ((double)M * p.pixel_A);
        const double fx = (double)(kx <= (M - 1) / 2 ? kx : kx - M) / ((double)M * p.pixel_A);
        const double ph = -M_PI * p.lambda_A * p.dz_A * (fy * fy + fx * fx);
        rows[(ky - k0) * M + kx] =
            make_float2((float)(std::cos(ph) / ((double)M * M)), (float)(std::sin(ph) / ((double)M * M)));
      }
    if ((e = cudaMemcpyAsync(d_h2 + (size_t)k0 * M, rows, 16 * M * sizeof(float2), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
  }
  // Everything that must start at zero is cleared here: the previous call's
  // contents stay in the scratch.
  if ((e = cudaMemcpyAsync(d_tw, tw, M * sizeof(float2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_hs, hs, M * sizeof(float2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_status, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_loss, 0, sizeof(double), st)) != cudaSuccess)
    return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));

  if (p.N == 0) {
    if (grad_obj && (e = cudaMemsetAsync(grad_obj, 0, sizeof(float2) * (size_t)p.S * p.H * p.W, st)) != cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
    if (grad_probe && (e = cudaMemsetAsync(grad_probe, 0, sizeof(float2) * MM, st)) != cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
  }
  const int2* pos = reinterpret_cast<const int2*>(pos_yx);
  if ((e = launch_check_positions(pos, p.N, M, p.H, p.W, d_status, st)) != cudaSuccess)
    return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));

  ChainArgs a{};
  a.pos = pos;
  a.probe = reinterpret_cast<const float2*>(probe);
  a.obj = reinterpret_cast<const float2*>(obj);
  a.meas = meas_I;
  a.S = p.S;
  a.H = p.H;
  a.W = p.W;
  a.tw = d_tw;
  a.hs = d_hs;
  a.h2 = d_h2;
  a.ws_n = chunk;
  a.ws_psi = ws_psi;
  a.ws_gphi = ws_gphi;
  a.ws_gp = ws_gp;
  a.loss_part = loss_part;
  a.status = d_status;
  const bool want_grad = grad_obj || grad_probe;
  for (int c0 = 0, ci = 0; c0 < p.N; c0 += chunk, ++ci) {
    const int n = p.N - c0 < chunk ? p.N - c0 : chunk;
    a.pos_begin = c0;
    a.n_pos = n;
    if ((e = launch_chain(M, want_grad ? MODE_GRAD : MODE_LOSS, a, st)) != cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
    if (grad_obj) {
      AccumArgs g{};
      g.pos = pos;
      g.pos_begin = c0;
      g.n_pos = n;
      g.M = M;
      g.S = p.S;
      g.H = p.H;
      g.W = p.W;
      g.tile_h = th;
      g.tile_w = tw_;
      g.probe = a.probe;
      g.ws_n = chunk;
      g.ws_psi = ws_psi;
      g.ws_gphi = ws_gphi;
      g.grad_obj = reinterpret_cast<float2*>(grad_obj);
      g.accumulate = ci > 0;
      if ((e = launch_accum_obj_grad(g, st)) != cudaSuccess) return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
    }
    if (grad_probe &&
        (e = launch_probe_grad(ws_gp, n, M, gp_part, kSplit, reinterpret_cast<float2*>(grad_probe), ci > 0, st)) !=
            cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
    if ((e = launch_loss_accum(loss_part, n, d_loss, ci > 0, st)) != cudaSuccess)
      return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
  }

  // The call is synchronous: it waits for the stream to report the status.
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(loss_out, d_loss, sizeof(double), cudaMemcpyDefault, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return noalloc_fail(PTYCHO_ERR_CUDA, cudaGetErrorString(e));
  if (status) return noalloc_fail(PTYCHO_ERR_POSITION, "a probe window lies outside the object");
  return PTYCHO_OK;
}
