// C-ABI of libptycho: plan management, argument validation and the host-side
// orchestration of the per-chunk kernel sequence.  See include/ptycho.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ptycho.h"
#include "internal.h"

using namespace ptycho;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(PTYCHO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Round to BF16 (nearest, ties to even) on the host.
uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float host_bf16_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Round to IEEE half (nearest, ties to even) on the host, with subnormals.
uint16_t host_f16(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const uint32_t fexp = (x >> 23) & 0xFFu;
  uint32_t mant = x & 0x7FFFFFu;
  if (fexp == 0xFFu) return (uint16_t)(sign | 0x7C00u | (mant ? 0x200u : 0u));
  int exp = (int)fexp - 127 + 15;
  if (exp >= 31) return (uint16_t)(sign | 0x7C00u);
  if (exp <= 0) {
    const int shift = 14 - exp;  // 24-bit significand -> subnormal units of 2^-24
    if (shift > 24) return (uint16_t)sign;
    mant |= 0x800000u;
    uint32_t q = mant >> shift;
    const uint32_t rem = mant & ((1u << shift) - 1u), halfway = 1u << (shift - 1);
    if (rem > halfway || (rem == halfway && (q & 1u))) ++q;
    return (uint16_t)(sign | q);
  }
  uint32_t q = mant >> 13;
  const uint32_t rem = mant & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (q & 1u))) {
    if (++q == 0x400u) {
      q = 0;
      if (++exp >= 31) return (uint16_t)(sign | 0x7C00u);
    }
  }
  return (uint16_t)(sign | ((uint32_t)exp << 10) | q);
}
float host_f16_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const int e = (h >> 10) & 0x1F;
  const uint32_t m = h & 0x3FFu;
  float v;
  if (e == 0) v = std::ldexp((float)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp((float)(m | 0x400u), e - 25);
  return sign ? -v : v;
}

// Tensor-core operand planes of the two transform matrices, computed in FP64:
//   K[m][n] = (1/M) sum_k h1(k) exp(+2 pi i k (m - n) / M)   (propagator, separable factor)
//   F[m][n] = exp(-2 pi i m n / M) / sqrt(M)                  (orthonormal DFT)
// Each entry is split into BF16 hi + lo for the real and imaginary parts;
// row m of a plane is 64 words, element 2c in the low half of word c.
std::vector<uint32_t> build_tc_planes(const ptycho_params& p, bool f16) {
  const int M = p.M;
  std::vector<uint32_t> out((size_t)2 * 4 * M * (M / 2));
  std::vector<double> h1r(M), h1i(M);
  for (int k = 0; k < M; ++k) {
    const double f = (double)(k <= (M - 1) / 2 ? k : k - M) / ((double)M * p.pixel_A);
    const double ph = -M_PI * p.lambda_A * p.dz_A * f * f;
    h1r[k] = std::cos(ph);
    h1i[k] = std::sin(ph);
  }
  const double two_pi = 6.283185307179586476925287;
  for (int which = 0; which < 2; ++which) {
    std::vector<double> cr((size_t)M * M), ci((size_t)M * M);
    for (int m = 0; m < M; ++m)
      for (int n = 0; n < M; ++n) {
        if (which == 0) {
          double sr = 0.0, si = 0.0;
          for (int k = 0; k < M; ++k) {
            const double a = two_pi * (double)k * (double)(m - n) / (double)M;
            const double c = std::cos(a), s = std::sin(a);
            sr += h1r[k] * c - h1i[k] * s;
            si += h1r[k] * s + h1i[k] * c;
          }
          cr[(size_t)m * M + n] = sr / M;
          ci[(size_t)m * M + n] = si / M;
        } else {
          const double a = -two_pi * (double)(((long long)m * n) % M) / (double)M;
          cr[(size_t)m * M + n] = std::cos(a) / std::sqrt((double)M);
          ci[(size_t)m * M + n] = std::sin(a) / std::sqrt((double)M);
        }
      }
    for (int part = 0; part < 2; ++part) {
      const std::vector<double>& src = part == 0 ? cr : ci;
      for (int m = 0; m < M; ++m)
        for (int c = 0; c < M / 2; ++c) {
          uint16_t hi[2], lo[2];
          for (int e = 0; e < 2; ++e) {
            const float x = (float)src[(size_t)m * M + 2 * c + e];
            if (f16) {
              hi[e] = host_f16(x);
              lo[e] = host_f16(x - host_f16_to_float(hi[e]));
            } else {
              hi[e] = host_bf16(x);
              lo[e] = host_bf16(x - host_bf16_to_float(hi[e]));
            }
          }
          const size_t base = ((size_t)which * 4 * M + (size_t)m) * (M / 2) + c;
          out[base + (size_t)(2 * part) * M * (M / 2)] = (uint32_t)hi[1] << 16 | hi[0];
          out[base + (size_t)(2 * part + 1) * M * (M / 2)] = (uint32_t)lo[1] << 16 | lo[0];
        }
    }
  }
  return out;
}

constexpr int64_t kDefaultWorkspace = 8ll << 30;
// Generic-window path: the most bytes of chunk waves (streamed by every pass)
#ifndef PTYCHO_GM_WAVE_BYTES
#define PTYCHO_GM_WAVE_BYTES (64ll << 20)
#endif
constexpr int kProbeSplit = 32;
constexpr int kNormParts = 512;

}  // namespace

struct ptycho_plan_s {
  ptycho_params p{};
  int device = 0;
  int sm_count = 0;
  int chunk = 0;             // positions per chunk
  int ckpt_L = 0;            // recompute segment length (0 = keep every wave)
  int64_t ws_bytes = 0;
  float2* d_tw = nullptr;     // [M]
  float2* d_hs = nullptr;     // [M]
  float2* d_h2 = nullptr;     // [M][M] (M = 64, 128)
  float2* ws_psi = nullptr;   // [S-1][chunk][M][M] (recompute: [K-2+L+1][chunk][M][M])
  float2* ws_gphi = nullptr;  // [S][chunk][M][M] (recompute: none)
  float2* ws_gp = nullptr;    // [chunk][M][M]
  float2* wv = nullptr;       // generic-window path: [chunk][M][M] waves of the chunk
  float2* gp_part = nullptr;  // [kProbeSplit][M][M]
  double* loss_part = nullptr;  // [chunk]
  double* d_scal = nullptr;   // [8]: 0 loss, 1 |gO|^2, 2 |gP|^2, 3 trial loss
  double* norm_part = nullptr;  // [kNormParts]
  int* d_status = nullptr;
  int* h_pos = nullptr;       // pinned, [N][2]
  double* h_scal = nullptr;   // pinned, [8]
  int* h_flag = nullptr;      // pinned, [1]: the device error word, read by the synchronous calls
  // gradient-descent step buffers (allocated on first use)
  float2* g_obj = nullptr;
  float2* g_probe = nullptr;
  uint32_t* d_cplanes = nullptr;  // BF16X3: [K, F][re_hi, re_lo, im_hi, im_lo][128][64] packed BF16 pairs
  // kernel timing: event pairs per kernel family, launch counters
  // side stream for the object-gradient accumulation of a chunk's full chain
  // waves while its partial last wave runs (fork/join by events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int wave = 0;               // chain blocks resident on the whole GPU at once
  // host-buffer entry point (allocated on first use): device copies of the
  // inputs and gradients, and a copy stream that uploads the intensities of
  // all but the first chain wave while that wave runs
  int32_t* x_pos = nullptr;
  float2* x_probe = nullptr;
  float2* x_obj = nullptr;
  float* x_meas = nullptr;
  float2* x_gO = nullptr;
  float2* x_gP = nullptr;
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_first = nullptr, ev_rest = nullptr;
  struct Mark {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  size_t n_marks = 0;
  ptycho_timing tm{};
};

namespace {

void free_plan(ptycho_plan pl) {
  if (!pl) return;
  for (auto& m : pl->marks) {
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  cudaFree(pl->d_tw);
  cudaFree(pl->d_hs);
  cudaFree(pl->d_h2);
  cudaFree(pl->ws_psi);
  cudaFree(pl->ws_gphi);
  cudaFree(pl->ws_gp);
  cudaFree(pl->wv);
  cudaFree(pl->gp_part);
  cudaFree(pl->loss_part);
  cudaFree(pl->d_scal);
  cudaFree(pl->norm_part);
  cudaFree(pl->d_status);
  cudaFree(pl->g_obj);
  cudaFree(pl->g_probe);
  cudaFree(pl->d_cplanes);
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  if (pl->side) cudaStreamDestroy(pl->side);
  cudaFree(pl->x_pos);
  cudaFree(pl->x_probe);
  cudaFree(pl->x_obj);
  cudaFree(pl->x_meas);
  cudaFree(pl->x_gO);
  cudaFree(pl->x_gP);
  if (pl->ev_first) cudaEventDestroy(pl->ev_first);
  if (pl->ev_rest) cudaEventDestroy(pl->ev_rest);
  if (pl->copy) cudaStreamDestroy(pl->copy);
  if (pl->h_pos) cudaFreeHost(pl->h_pos);
  if (pl->h_scal) cudaFreeHost(pl->h_scal);
  if (pl->h_flag) cudaFreeHost(pl->h_flag);
  delete pl;
}

template <class T>
int dev_alloc(T** p, size_t count, const char* what) {
  if (count == 0) {
    *p = nullptr;
    return PTYCHO_OK;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(PTYCHO_ERR_NOMEM, std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
  }
  return PTYCHO_OK;
}

bool fused_window(int M) { return M == 64 || M == 128; }

int validate_params(const ptycho_params& p) {
  if (!fused_window(p.M) && !(p.precision == PTYCHO_FP32 && gm_supported(p.M, nullptr)))
    return fail(PTYCHO_ERR_UNSUPPORTED,
                "probe window M must be 64 or 128, or (FP32) a product of powers of 2 and 3 in [8, 4096]");
  if (p.S < 1) return fail(PTYCHO_ERR_ARG, "S must be >= 1");
  if (p.H < p.M || p.W < p.M) return fail(PTYCHO_ERR_ARG, "object must be at least M x M");
  if (p.N < 0) return fail(PTYCHO_ERR_ARG, "N must be >= 0");
  if (p.precision != PTYCHO_FP32 && p.precision != PTYCHO_BF16X3 && p.precision != PTYCHO_FP16X3)
    return fail(PTYCHO_ERR_UNSUPPORTED, "precision must be PTYCHO_FP32, PTYCHO_BF16X3 or PTYCHO_FP16X3");
  if (p.precision != PTYCHO_FP32 && p.M != 128)
    return fail(PTYCHO_ERR_UNSUPPORTED, "the tensor-core precisions support M = 128 only");
  if (p.precision != PTYCHO_FP32 && p.ckpt_every > 0 && p.ckpt_every < p.S)
    return fail(PTYCHO_ERR_UNSUPPORTED, "the tensor-core precisions do not support the recompute mode");
  if (!(p.pixel_A > 0) || !std::isfinite(p.lambda_A) || !std::isfinite(p.dz_A))
    return fail(PTYCHO_ERR_ARG, "bad propagator parameters");
  if (p.workspace_bytes < 0) return fail(PTYCHO_ERR_ARG, "workspace_bytes must be >= 0");
  const int th = p.tile_h ? p.tile_h : kDefaultTile, tw = p.tile_w ? p.tile_w : kDefaultTile;
  if (th < 1 || tw < 1 || th * tw > 8192) return fail(PTYCHO_ERR_ARG, "tile_h * tile_w must be in [1, 8192]");
  if ((int64_t)p.S * p.H * p.W > (int64_t)1 << 34) return fail(PTYCHO_ERR_ARG, "object too large");
  if (p.ckpt_every < 0 && p.ckpt_every != PTYCHO_CKPT_AUTO)
    return fail(PTYCHO_ERR_ARG, "ckpt_every must be >= 0 or PTYCHO_CKPT_AUTO");
  return PTYCHO_OK;
}

int check_windows(const ptycho_params& p, const int32_t* h_pos);

// The error a non-zero device error word stands for.
int status_fail(int h) {
  if (h == PTYCHO_ERR_TIMEOUT) return fail(h, "a bounded tensor-core wait gave up on the device");
  if (h == PTYCHO_ERR_UNSUPPORTED) return fail(h, "a wave value left the FP16 range (|x| >= 60000)");
  return fail(h, "a probe window outside the object was skipped on the device");
}

// Positions check on the host (pinned copy) unless the plan asks for the
// asynchronous device-side check only.
int check_positions(ptycho_plan pl, const int32_t* pos, cudaStream_t st) {
  const ptycho_params& p = pl->p;
  if (p.N == 0) return PTYCHO_OK;
  if (!is_device_ptr(pos)) return fail(PTYCHO_ERR_ARG, "pos_yx must be a device pointer");
  if (!aligned(pos, 8)) return fail(PTYCHO_ERR_ARG, "pos_yx must be 8-byte aligned");
  if (p.flags & PTYCHO_FLAG_ASYNC_CHECK) return PTYCHO_OK;
  CUDA_TRY(cudaMemcpyAsync(pl->h_pos, pos, sizeof(int32_t) * 2 * (size_t)p.N, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return check_windows(p, pl->h_pos);
}

// Every window inside the object: 0 <= y <= H - M, 0 <= x <= W - M.
int check_windows(const ptycho_params& p, const int32_t* h_pos) {
  for (int i = 0; i < p.N; ++i) {
    const int y = h_pos[2 * i], x = h_pos[2 * i + 1];
    if (y < 0 || x < 0 || y > p.H - p.M || x > p.W - p.M) {
      char buf[160];
      snprintf(buf, sizeof buf, "position %d (y=%d, x=%d) puts the %dx%d window outside the %dx%d object", i, y, x,
               p.M, p.M, p.H, p.W);
      return fail(PTYCHO_ERR_POSITION, buf);
    }
  }
  return PTYCHO_OK;
}

int check_array(const void* ptr, const char* name, bool required) {
  if (!ptr) return required ? fail(PTYCHO_ERR_ARG, std::string(name) + " is NULL") : PTYCHO_OK;
  if (!is_device_ptr(ptr)) return fail(PTYCHO_ERR_ARG, std::string(name) + " must be a device pointer");
  if (!aligned(ptr, 8)) return fail(PTYCHO_ERR_ARG, std::string(name) + " must be 8-byte aligned");
  return PTYCHO_OK;
}

enum Kind { K_CHAIN = 0, K_ACCUM = 1, K_PROBE = 2, K_OTHER = 3 };

// Run `launch` (which enqueues `n_kernels` kernels on st) between two CUDA
// events when the plan records timings; always count the launches.
template <class F>
int timed(ptycho_plan pl, int kind, int n_kernels, cudaStream_t st, F&& launch) {
  const bool rec = (pl->p.flags & PTYCHO_FLAG_TIMING) != 0;
  ptycho_plan_s::Mark* m = nullptr;
  if (rec) {
    if (pl->n_marks == pl->marks.size()) {
      ptycho_plan_s::Mark nm{kind, nullptr, nullptr};
      CUDA_TRY(cudaEventCreate(&nm.start));
      CUDA_TRY(cudaEventCreate(&nm.stop));
      pl->marks.push_back(nm);
    }
    m = &pl->marks[pl->n_marks++];
    m->kind = kind;
    CUDA_TRY(cudaEventRecord(m->start, st));
  }
  CUDA_TRY(launch());
  if (rec) CUDA_TRY(cudaEventRecord(m->stop, st));
  pl->tm.launches += n_kernels;
  if (kind == K_CHAIN) pl->tm.chain_launches += n_kernels;
  if (kind == K_ACCUM) pl->tm.accum_launches += n_kernels;
  return PTYCHO_OK;
}

#define TIMED_ON(stream, kind, nk, expr)                                      \
  do {                                                                        \
    int rc_ = timed(pl, kind, nk, stream, [&]() -> cudaError_t { return expr; }); \
    if (rc_) return rc_;                                                      \
  } while (0)
#define TIMED(kind, nk, expr) TIMED_ON(st, kind, nk, expr)

ChainArgs base_args(ptycho_plan pl, const int32_t* pos, const ptycho_c64* probe, const ptycho_c64* obj,
                    const float* meas) {
  ChainArgs a{};
  a.pos = reinterpret_cast<const int2*>(pos);
  a.probe = reinterpret_cast<const float2*>(probe);
  a.obj = reinterpret_cast<const float2*>(obj);
  a.meas = meas;
  a.S = pl->p.S;
  a.H = pl->p.H;
  a.W = pl->p.W;
  a.tw = pl->d_tw;
  a.hs = pl->d_hs;
  a.h2 = pl->d_h2;
  a.ws_n = pl->chunk;
  a.ckpt_L = pl->ckpt_L;
  a.ws_psi = pl->ws_psi;
  a.ws_gphi = pl->ws_gphi;
  a.ws_gp = pl->ws_gp;
  a.loss_part = pl->loss_part;
  a.status = pl->d_status;
  a.selftest_timeout = (pl->p.flags & PTYCHO_FLAG_SELFTEST_TIMEOUT) ? 1 : 0;
  return a;
}

// Object-gradient accumulation (every wave kept) of positions
// [c0 + off, c0 + off + n) of the current chunk, whose workspace slots start
// at off.
int accum_part(ptycho_plan pl, const int32_t* pos, const ptycho_c64* probe, float2* grad_obj, int c0, int off,
               int n, int accumulate, cudaStream_t st) {
  const ptycho_params& p = pl->p;
  const size_t MM = (size_t)p.M * p.M;
  AccumArgs g{};
  g.pos = reinterpret_cast<const int2*>(pos);
  g.pos_begin = c0 + off;
  g.n_pos = n;
  g.M = p.M;
  g.S = p.S;
  g.H = p.H;
  g.W = p.W;
  g.tile_h = p.tile_h ? p.tile_h : kDefaultTile;
  g.tile_w = p.tile_w ? p.tile_w : kDefaultTile;
  g.probe = reinterpret_cast<const float2*>(probe);
  g.ws_n = pl->chunk;
  g.ws_psi = pl->ws_psi + (size_t)off * MM;
  g.ws_gphi = pl->ws_gphi + (size_t)off * MM;
  g.grad_obj = grad_obj;
  g.accumulate = accumulate;
  TIMED(K_ACCUM, 1, launch_accum_obj_grad(g, st));
  return PTYCHO_OK;
}

// F (and optionally gradients) at (probe + probe_step*probe_dir, obj + obj_step*obj_dir);
// the loss lands in pl->d_scal[slot].  With rest_ready, only the intensities
// of the first n_first positions are ready when the call starts: the chain of
// those positions is launched first, then st waits for rest_ready.
int run_loss_grad(ptycho_plan pl, const int32_t* pos, const ptycho_c64* probe, const ptycho_c64* obj,
                  const float* meas, float2* grad_obj, float2* grad_probe, int slot, const float2* obj_dir,
                  float obj_step, const float2* probe_dir, float probe_step, cudaStream_t st,
                  int n_first = 0, cudaEvent_t rest_ready = nullptr) {
  const ptycho_params& p = pl->p;
  const bool want_grad = grad_obj || grad_probe;
  if (p.N == 0) {
    CUDA_TRY(cudaMemsetAsync(pl->d_scal + slot, 0, sizeof(double), st));
    if (grad_obj) CUDA_TRY(cudaMemsetAsync(grad_obj, 0, sizeof(float2) * (size_t)p.S * p.H * p.W, st));
    if (grad_probe) CUDA_TRY(cudaMemsetAsync(grad_probe, 0, sizeof(float2) * (size_t)p.M * p.M, st));
    return PTYCHO_OK;
  }
  ChainArgs a = base_args(pl, pos, probe, obj, meas);
  a.obj_dir = obj_dir;
  a.obj_step = obj_step;
  a.probe_dir = probe_dir;
  a.probe_step = probe_step;
  const ChainMode mode = !want_grad ? MODE_LOSS : (pl->ckpt_L ? MODE_GRAD_RC : MODE_GRAD);
  const size_t MM = (size_t)p.M * p.M;
  // Positions [off, off + n) of the current chunk (workspace slots from off).
  auto sub = [&](const ChainArgs& ca, int off, int n) {
    ChainArgs r = ca;
    r.pos_begin = ca.pos_begin + off;
    r.n_pos = n;
    r.ws_psi = pl->ws_psi + (size_t)off * MM;
    r.ws_gphi = pl->ws_gphi ? pl->ws_gphi + (size_t)off * MM : nullptr;
    r.ws_gp = pl->ws_gp + (size_t)off * MM;
    r.loss_part = pl->loss_part + off;
    return r;
  };
  auto launch_chain_for = [&](const ChainArgs& ca) -> int {
    int gm_launches = 0;
    if (pl->wv) {
      TIMED(K_CHAIN, 0, launch_chain_gm(mode, ca, pl->wv, p.M, &gm_launches, st));
      pl->tm.launches += gm_launches;
      pl->tm.chain_launches += 1;
    } else if (p.precision != PTYCHO_FP32) {
      TIMED(K_CHAIN, 1, launch_chain_tc(mode, ca, pl->d_cplanes, p.precision == PTYCHO_FP16X3, st));
    } else {
      TIMED(K_CHAIN, 1, launch_chain(p.M, mode, ca, st));
    }
    pl->tm.chain_positions += ca.n_pos;
    return PTYCHO_OK;
  };
  // Recompute mode: K segments of L slices; segment j's patches sit in the
  // L workspace slots from K-2 (see chain_kernels.cu).
  const bool recompute = want_grad && pl->ckpt_L > 0;
  const int rcL = pl->ckpt_L, rcK = recompute ? (p.S + rcL - 1) / rcL : 0;
  // Object-gradient accumulation of positions [c0 + off, c0 + off + n) of
  // the chunk, whose workspace slots start at off; in recompute mode, of the
  // slices of segment j.
  auto accum_for = [&](int c0, int off, int n, int accumulate, cudaStream_t on, int j = -1) -> int {
    AccumArgs g{};
    g.pos = a.pos;
    g.pos_begin = c0 + off;
    g.n_pos = n;
    g.M = p.M;
    g.S = p.S;
    g.H = p.H;
    g.W = p.W;
    g.tile_h = p.tile_h ? p.tile_h : kDefaultTile;
    g.tile_w = p.tile_w ? p.tile_w : kDefaultTile;
    g.probe = a.probe;
    g.ws_n = pl->chunk;
    g.ws_psi = pl->ws_psi + (size_t)off * MM;
    g.ws_gphi = pl->ws_gphi ? pl->ws_gphi + (size_t)off * MM : nullptr;
    g.grad_obj = grad_obj;
    g.accumulate = accumulate;
    if (j >= 0) {  // recompute segment j: the segment's slots
      if (pl->wv) {  // generic path: waves psi_s and exit-wave gradients g_phi_s
        g.ws_psi = pl->ws_psi + ((size_t)(rcK - 2) * pl->chunk + off) * MM;
      } else {       // register-resident path: finished patches over the waves
        g.ws_gphi = pl->ws_psi + ((size_t)(rcK - 2) * pl->chunk + off) * MM;
        g.patch_mode = 1;
      }
      g.seg_slots = 1;
      g.s_begin = j * rcL;
      g.n_slices = (j == rcK - 1 ? p.S : g.s_begin + rcL) - g.s_begin;
    }
    TIMED_ON(on, K_ACCUM, 1, launch_accum_obj_grad(g, on));
    return PTYCHO_OK;
  };
  for (int c0 = 0, ci = 0; c0 < p.N; c0 += pl->chunk, ++ci) {
    const int n = p.N - c0 < pl->chunk ? p.N - c0 : pl->chunk;
    // A chunk whose chain ends in a partial wave is launched as its full
    // waves and the tail: the accumulation of the full waves then runs on the
    // side stream, on the SMs the tail leaves idle.  The tail's workspace
    // slots follow the full waves', and its accumulation is added second, so
    // the summation order is fixed.
    const int tail =
        (grad_obj && !recompute && !pl->wv && pl->side && pl->wave > 0 && n > pl->wave) ? n % pl->wave : 0;
    const int n1 = n - tail;
    a.pos_begin = c0;
    a.n_pos = n1;
    int rc;
    if (rest_ready && ci == 0) {
      const int nf = n_first < n1 ? n_first : n1;
      if ((rc = launch_chain_for(sub(a, 0, nf))) != PTYCHO_OK) return rc;
      CUDA_TRY(cudaStreamWaitEvent(st, rest_ready, 0));
      if (n1 > nf && (rc = launch_chain_for(sub(a, nf, n1 - nf))) != PTYCHO_OK) return rc;
    } else if ((rc = launch_chain_for(a)) != PTYCHO_OK) {
      return rc;
    }
    if (recompute) {
      // The first launch differentiated the last segment; each later one
      // rebuilds and differentiates the segment before it, whose patches
      // overwrite the previous segment's: accumulate each before the next.
      for (int j = rcK - 1; j >= 0; --j) {
        if (j < rcK - 1) {
          ChainArgs sa = a;
          sa.n_pos = n;
          sa.seg = j;
          if (pl->wv) {
            int gm_launches = 0;
            TIMED(K_CHAIN, 0, launch_chain_gm(MODE_RC_SEG, sa, pl->wv, p.M, &gm_launches, st));
            pl->tm.launches += gm_launches;
            pl->tm.chain_launches += 1;
          } else {
            TIMED(K_CHAIN, 1, launch_chain(p.M, MODE_RC_SEG, sa, st));
          }
          pl->tm.chain_positions += n;
        }
        if (grad_obj && (rc = accum_for(c0, 0, n, ci > 0, st, j)) != PTYCHO_OK) return rc;
      }
    } else if (tail) {
      CUDA_TRY(cudaEventRecord(pl->ev_fork, st));
      if ((rc = launch_chain_for(sub(a, n1, tail))) != PTYCHO_OK) return rc;
      CUDA_TRY(cudaStreamWaitEvent(pl->side, pl->ev_fork, 0));
      if ((rc = accum_for(c0, 0, n1, ci > 0, pl->side)) != PTYCHO_OK) return rc;
      CUDA_TRY(cudaEventRecord(pl->ev_join, pl->side));
      CUDA_TRY(cudaStreamWaitEvent(st, pl->ev_join, 0));
      if ((rc = accum_for(c0, n1, tail, 1, st)) != PTYCHO_OK) return rc;
    } else if (grad_obj) {
      if ((rc = accum_for(c0, 0, n, ci > 0, st)) != PTYCHO_OK) return rc;
    }
    if (grad_probe)
      TIMED(K_PROBE, 2, launch_probe_grad(pl->ws_gp, n, p.M, pl->gp_part, kProbeSplit, grad_probe, ci > 0, st));
    TIMED(K_OTHER, 1, launch_loss_accum(pl->loss_part, n, pl->d_scal + slot, ci > 0, st));
  }
  return PTYCHO_OK;
}

int deliver_loss(ptycho_plan pl, int slot, double* loss_out, cudaStream_t st) {
  if (!loss_out) return PTYCHO_OK;
  if (is_device_ptr(loss_out)) {
    CUDA_TRY(cudaMemcpyAsync(loss_out, pl->d_scal + slot, sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    CUDA_TRY(cudaMemcpyAsync(pl->h_scal + slot, pl->d_scal + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *loss_out = pl->h_scal[slot];
  }
  return PTYCHO_OK;
}

}  // namespace

extern "C" {

const char* ptycho_last_error(void) { return g_last_error.c_str(); }

const char* ptycho_version(void) { return "libptycho 0.1 (sm_103a, FP32 register-pass FFT chain)"; }

int ptycho_plan_create(ptycho_plan* out, const ptycho_params* params) {
  g_last_error.clear();
  if (!out || !params) return fail(PTYCHO_ERR_ARG, "plan and params must be non-NULL");
  *out = nullptr;
  int rc = validate_params(*params);
  if (rc) return rc;
  ptycho_plan pl = new (std::nothrow) ptycho_plan_s;
  if (!pl) return fail(PTYCHO_ERR_NOMEM, "host allocation failed");
  pl->p = *params;
  const ptycho_params& p = pl->p;
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaGetDevice");
  }
  cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
  if ((fused_window(p.M) && (e = chain_prepare(p.M)) != cudaSuccess) ||
      (!fused_window(p.M) && (e = gm_prepare(p.M)) != cudaSuccess) ||
      (p.precision != PTYCHO_FP32 && (e = chain_tc_prepare()) != cudaSuccess)) {
    delete pl;
    return cuda_fail(e, "cudaFuncSetAttribute");
  }

  // Tables in FP64 on the host, rounded once to FP32.
  const int M = p.M;
  std::vector<float2> tw(M), hs(M);
  const double two_pi = 6.283185307179586476925287;
  for (int k = 0; k < M; ++k) {
    const double ang = -two_pi * (double)k / (double)M;
    tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    // fftfreq(M, pixel): k/(M*pixel) for k <= (M-1)/2, (k-M)/(M*pixel) otherwise (odd M too)
    const double f = (double)(k <= (M - 1) / 2 ? k : k - M) / ((double)M * p.pixel_A);
    const double ph = -M_PI * p.lambda_A * p.dz_A * f * f;
    hs[k] = make_float2((float)(std::cos(ph) / M), (float)(std::sin(ph) / M));
  }
  // The full propagator h(ky) h(kx) / M^2 for the register-resident kernels.
  std::vector<float2> h2;
  if (fused_window(M)) {
    h2.resize((size_t)M * M);
    for (int ky = 0; ky < M; ++ky)
      for (int kx = 0; kx < M; ++kx) {
        const double fy = (double)(ky <= (M - 1) / 2 ? ky : ky - M) / ((double)M * p.pixel_A);
        const double fx = (double)(kx <= (M - 1) / 2 ? kx : kx - M) / ((double)M * p.pixel_A);
        const double ph = -M_PI * p.lambda_A * p.dz_A * (fy * fy + fx * fx);
        h2[(size_t)ky * M + kx] =
            make_float2((float)(std::cos(ph) / ((double)M * M)), (float)(std::sin(ph) / ((double)M * M)));
      }
  }

  // Workspace per position in flight (gradient mode).
  const size_t MM = (size_t)M * M;
  int ckpt_req = p.ckpt_every;
  if (ckpt_req == PTYCHO_CKPT_AUTO) {  // K = ceil(sqrt(S)) checkpoints, interval ceil(S / K)
    int K = 1;
    while (K * K < p.S) ++K;
    ckpt_req = (p.S + K - 1) / K;
  }
  pl->ckpt_L = (ckpt_req > 0 && ckpt_req < p.S && p.precision == PTYCHO_FP32) ? ckpt_req : 0;
  const bool gm = !fused_window(M);
  // Recompute mode keeps K-2 checkpoints, one segment's L waves (then
  // patches) and the parked adjoint state: K + L - 1 waves whatever S is for
  // given K and L (about 2 sqrt(S) with the automatic choice), against
  // 2S - 1 when every wave is kept.  The generic-window path keeps the
  // segment's L exit-wave gradients beside its waves (and its wave buffer).
  const int K = pl->ckpt_L ? (p.S + pl->ckpt_L - 1) / pl->ckpt_L : 0;
  const size_t psi_slots = pl->ckpt_L ? (size_t)(K - 2 + pl->ckpt_L + 1) : (size_t)(p.S - 1);
  const size_t gphi_slots = pl->ckpt_L ? (gm ? (size_t)pl->ckpt_L : 0) : (size_t)p.S;
  const size_t per_pos =
      (psi_slots + gphi_slots + (gm ? 1 : 0)) * MM * sizeof(float2) + MM * sizeof(float2) + sizeof(double);
  const int64_t cap = p.workspace_bytes ? p.workspace_bytes : kDefaultWorkspace;
  int64_t chunk = cap / (int64_t)per_pos;
  // generic-window path: keep the chunk's waves (streamed by every FFT pass)
  // within about half of the L2
  if (gm && chunk > 1) {
    const int64_t l2cap = (int64_t)PTYCHO_GM_WAVE_BYTES / (int64_t)(MM * sizeof(float2));
    if (chunk > l2cap) chunk = l2cap > 1 ? l2cap : 1;
  }
  if (chunk < 1) {
    delete pl;
    return fail(PTYCHO_ERR_NOMEM, "workspace_bytes too small for one position");
  }
  const int n = p.N > 0 ? p.N : 1;
  if (chunk >= n) {
    chunk = n;
  } else {
    const int blocks_per_wave = pl->sm_count * (M == 128 ? 1 : 4);
    if (chunk > blocks_per_wave) chunk -= chunk % blocks_per_wave;
  }
  pl->chunk = (int)chunk;
  // Chain blocks resident on the GPU at once: the occupancy of the FP32
  // gradient kernel, or one split-product block per SM (all of tensor memory).
  if (!gm) pl->wave = pl->sm_count * (p.precision == PTYCHO_FP32 ? chain_blocks_per_sm(M) : 1);

  rc = PTYCHO_OK;
  if (!rc) rc = dev_alloc(&pl->d_tw, M, "twiddles");
  if (!rc) rc = dev_alloc(&pl->d_hs, M, "propagator");
  if (!rc) rc = dev_alloc(&pl->d_h2, h2.size(), "propagator table");
  if (!rc) rc = dev_alloc(&pl->ws_psi, (size_t)pl->chunk * psi_slots * MM, "wave workspace");
  if (!rc) rc = dev_alloc(&pl->ws_gphi, (size_t)pl->chunk * gphi_slots * MM, "adjoint workspace");
  if (!rc) rc = dev_alloc(&pl->ws_gp, (size_t)pl->chunk * MM, "probe-gradient workspace");
  if (!rc && gm) rc = dev_alloc(&pl->wv, (size_t)pl->chunk * MM, "generic-window wave buffer");
  if (!rc) rc = dev_alloc(&pl->gp_part, (size_t)kProbeSplit * MM, "probe-gradient partials");
  if (!rc) rc = dev_alloc(&pl->loss_part, (size_t)pl->chunk, "loss partials");
  if (!rc) rc = dev_alloc(&pl->d_scal, 8, "scalars");
  if (!rc) rc = dev_alloc(&pl->norm_part, kNormParts, "norm partials");
  if (!rc) rc = dev_alloc(&pl->d_status, 1, "status");
  std::vector<uint32_t> planes;
  if (!rc && p.precision != PTYCHO_FP32) {
    planes = build_tc_planes(p, p.precision == PTYCHO_FP16X3);
    rc = dev_alloc(&pl->d_cplanes, planes.size(), "tensor-core operand planes");
  }
  if (!rc && !gm &&
      ((e = cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
       (e = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming)) != cudaSuccess))
    rc = cuda_fail(e, "side stream");
  if (rc) {
    free_plan(pl);
    return rc;
  }
  if (!planes.empty() &&
      (e = cudaMemcpy(pl->d_cplanes, planes.data(), planes.size() * sizeof(uint32_t), cudaMemcpyHostToDevice)) !=
          cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "plane upload");
  }
  if (cudaMallocHost(&pl->h_pos, sizeof(int32_t) * 2 * (size_t)n) != cudaSuccess ||
      cudaMallocHost(&pl->h_scal, sizeof(double) * 8) != cudaSuccess ||
      cudaMallocHost(&pl->h_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_plan(pl);
    return fail(PTYCHO_ERR_NOMEM, "pinned host allocation failed");
  }
  pl->ws_bytes = (int64_t)pl->chunk * (int64_t)per_pos;
  if ((e = cudaMemcpy(pl->d_tw, tw.data(), M * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(pl->d_hs, hs.data(), M * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!h2.empty() &&
       (e = cudaMemcpy(pl->d_h2, h2.data(), h2.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemset(pl->d_status, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(pl->d_scal, 0, 8 * sizeof(double))) != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "table upload");
  }
  *out = pl;
  return PTYCHO_OK;
}

int ptycho_plan_destroy(ptycho_plan plan) {
  g_last_error.clear();
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  cudaDeviceSynchronize();
  free_plan(plan);
  return PTYCHO_OK;
}

int ptycho_plan_info(ptycho_plan plan, int32_t* chunk_positions, int64_t* workspace_bytes) {
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  if (chunk_positions) *chunk_positions = plan->chunk;
  if (workspace_bytes) *workspace_bytes = plan->ws_bytes;
  return PTYCHO_OK;
}

int ptycho_plan_status(ptycho_plan plan) {
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  int h = 0;
  CUDA_TRY(cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(plan->d_status, 0, sizeof(int)));
  return h ? status_fail(h) : PTYCHO_OK;
}

int ptycho_plan_timing(ptycho_plan plan, ptycho_timing* out, int32_t reset) {
  g_last_error.clear();
  if (!plan || !out) return fail(PTYCHO_ERR_ARG, "plan and out must be non-NULL");
  ptycho_timing t = plan->tm;
  t.chain_ms = t.accum_ms = t.probe_ms = t.other_ms = 0.0;
  for (size_t i = 0; i < plan->n_marks; ++i) {
    const auto& m = plan->marks[i];
    CUDA_TRY(cudaEventSynchronize(m.stop));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, m.start, m.stop));
    double* dst = m.kind == K_CHAIN ? &t.chain_ms : m.kind == K_ACCUM ? &t.accum_ms
                : m.kind == K_PROBE ? &t.probe_ms : &t.other_ms;
    *dst += ms;
  }
  *out = t;
  if (reset) {
    plan->tm = ptycho_timing{};
    plan->n_marks = 0;
  }
  return PTYCHO_OK;
}

int ptycho_forward(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe, const ptycho_c64* obj,
                   ptycho_c64* psi_out, float* intens_out, void* stream) {
  g_last_error.clear();
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  if (!psi_out && !intens_out) return fail(PTYCHO_ERR_ARG, "psi_out and intens_out are both NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc;
  if ((rc = check_array(probe, "probe", true)) || (rc = check_array(obj, "obj", true)) ||
      (rc = check_array(psi_out, "psi_out", false)) || (rc = check_array(intens_out, "intens_out", false)))
    return rc;
  if ((rc = check_positions(plan, pos_yx, st))) return rc;
  const ptycho_params& p = plan->p;
  ChainArgs a = base_args(plan, pos_yx, probe, obj, nullptr);
  a.psi_out = reinterpret_cast<float2*>(psi_out);
  a.int_out = intens_out;
  // The register-resident and tensor-core kernels need no workspace in this
  // mode; the generic-window path stages the chunk's waves in wv, which holds
  // plan->chunk positions.
  const int step = plan->wv ? plan->chunk : 1 << 20;
  ptycho_plan pl = plan;
  for (int c0 = 0; c0 < p.N; c0 += step) {
    a.pos_begin = c0;
    a.n_pos = p.N - c0 < step ? p.N - c0 : step;
    int gm_launches = 0;
    if (pl->wv) {
      TIMED(K_CHAIN, 0, launch_chain_gm(MODE_FORWARD, a, pl->wv, p.M, &gm_launches, st));
      pl->tm.launches += gm_launches;
      pl->tm.chain_launches += 1;
    } else if (p.precision != PTYCHO_FP32)
      TIMED(K_CHAIN, 1, launch_chain_tc(MODE_FORWARD, a, pl->d_cplanes, p.precision == PTYCHO_FP16X3, st));
    else
      TIMED(K_CHAIN, 1, launch_chain(p.M, MODE_FORWARD, a, st));
    pl->tm.chain_positions += a.n_pos;
  }
  return PTYCHO_OK;
}

}  // extern "C"

namespace {

int loss_grad_impl(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe, const ptycho_c64* obj,
                   const float* meas_I, double* loss_out, ptycho_c64* grad_obj, ptycho_c64* grad_probe,
                   cudaStream_t st) {
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  int rc;
  if ((rc = check_array(probe, "probe", true)) || (rc = check_array(obj, "obj", true)) ||
      (rc = check_array(meas_I, "meas_I", plan->p.N > 0)) || (rc = check_array(grad_obj, "grad_obj", false)) ||
      (rc = check_array(grad_probe, "grad_probe", false)))
    return rc;
  if ((rc = check_positions(plan, pos_yx, st))) return rc;
  rc = run_loss_grad(plan, pos_yx, probe, obj, meas_I, reinterpret_cast<float2*>(grad_obj),
                     reinterpret_cast<float2*>(grad_probe), 0, nullptr, 0.f, nullptr, 0.f, st);
  if (rc) return rc;
  return deliver_loss(plan, 0, loss_out, st);
}

int step_impl(ptycho_plan plan, const int32_t* pos_yx, ptycho_c64* probe, ptycho_c64* obj, const float* meas_I,
              double alpha_obj, double alpha_probe, int32_t line_search, double* loss_out, double* t_out,
              cudaStream_t st) {
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  if (!std::isfinite(alpha_obj) || !std::isfinite(alpha_probe))
    return fail(PTYCHO_ERR_ARG, "step sizes must be finite");
  const ptycho_params& p = plan->p;
  int rc;
  if ((rc = check_array(probe, "probe", true)) || (rc = check_array(obj, "obj", true)) ||
      (rc = check_array(meas_I, "meas_I", p.N > 0)))
    return rc;
  if ((rc = check_positions(plan, pos_yx, st))) return rc;
  const size_t nO = (size_t)p.S * p.H * p.W, nP = (size_t)p.M * p.M;
  if (!plan->g_obj && (rc = dev_alloc(&plan->g_obj, nO, "step object gradient"))) return rc;
  if (!plan->g_probe && (rc = dev_alloc(&plan->g_probe, nP, "step probe gradient"))) return rc;
  rc = run_loss_grad(plan, pos_yx, probe, obj, meas_I, plan->g_obj, plan->g_probe, 0, nullptr, 0.f, nullptr, 0.f, st);
  if (rc) return rc;
  if ((rc = deliver_loss(plan, 0, loss_out, st))) return rc;
  float2* O = reinterpret_cast<float2*>(obj);
  float2* P = reinterpret_cast<float2*>(probe);
  ptycho_plan pl = plan;
  double t = 1.0;
  if (line_search) {
    TIMED(K_OTHER, 2, launch_norm2(plan->g_obj, nO, plan->norm_part, kNormParts, plan->d_scal, 1, st));
    TIMED(K_OTHER, 2, launch_norm2(plan->g_probe, nP, plan->norm_part, kNormParts, plan->d_scal, 2, st));
    CUDA_TRY(cudaMemcpyAsync(plan->h_scal, plan->d_scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const double F0 = plan->h_scal[0];
    const double dec = alpha_obj * plan->h_scal[1] + alpha_probe * plan->h_scal[2];
    bool accepted = false;
    for (int k = 0; k <= 20; ++k) {
      rc = run_loss_grad(plan, pos_yx, probe, obj, meas_I, nullptr, nullptr, 3, plan->g_obj,
                         (float)(-t * alpha_obj), plan->g_probe, (float)(-t * alpha_probe), st);
      if (rc) return rc;
      CUDA_TRY(cudaMemcpyAsync(plan->h_scal + 3, plan->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      if (plan->h_scal[3] <= F0 - 1e-4 * t * dec) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) t = 0.0;
  }
  if (t > 0.0) {
    TIMED(K_OTHER, 1, launch_axpy(O, plan->g_obj, O, -t * alpha_obj, nO, st));
    TIMED(K_OTHER, 1, launch_axpy(P, plan->g_probe, P, -t * alpha_probe, nP, st));
  }
  if (t_out) *t_out = t;
  return PTYCHO_OK;
}

// Run fn(problem) for every problem, in order, on st.  (Running the problems
// concurrently on their own streams was measured slower on the batched
// workload: the generic-window problems size their chunks to the L2 and then
// compete for it.)  Returns the first error, tagged with the problem's index.
template <class F>
int run_multi(const ptycho_problem* probs, int32_t n, F&& fn) {
  if (n < 0 || (n > 0 && !probs)) return fail(PTYCHO_ERR_ARG, "problems must be non-NULL and n >= 0");
  for (int32_t i = 0; i < n; ++i) {
    if (!probs[i].plan) return fail(PTYCHO_ERR_ARG, "problem " + std::to_string(i) + ": plan is NULL");
    if (probs[i].loss_out && !is_device_ptr(probs[i].loss_out))
      return fail(PTYCHO_ERR_ARG, "problem " + std::to_string(i) + ": loss_out must be a device pointer or NULL");
    for (int32_t j = 0; j < i; ++j)
      if (probs[j].plan == probs[i].plan)
        return fail(PTYCHO_ERR_ARG, "problems " + std::to_string(j) + " and " + std::to_string(i) +
                                        " share a plan");
  }
  for (int32_t i = 0; i < n; ++i) {
    const int rc = fn(probs[i]);
    if (rc) {
      g_last_error = "problem " + std::to_string(i) + ": " + g_last_error;
      return rc;
    }
  }
  return PTYCHO_OK;
}

// Problems whose chains the multi-problem launch takes: FP32, M = 64 or 128,
// every wave kept, at least one position.
bool fusable(ptycho_plan pl) {
  return pl->p.precision == PTYCHO_FP32 && fused_window(pl->p.M) && pl->ckpt_L == 0 && !pl->wv && pl->p.N > 0;
}

// The batched workload's register-resident problems, one iteration: for each
// window (64, 128), round r launches the chains of chunk r of every problem
// that has one in a single kernel (up to kMultiChainMax problems per launch),
// then runs each problem's reductions of that chunk exactly as its own call
// would (the same kernels, inputs and summation order, so the results are
// bit-identical to the single-problem calls).  With `step`, the gradients go
// to the plans' step buffers and the fixed-step update follows.
int run_multi_fused(const ptycho_problem* probs, const std::vector<int>& idx, bool step, double a_o, double a_p,
                    cudaStream_t st) {
  struct Item {
    int i;
    ptycho_plan pl;
    float2* gO;
    float2* gP;
  };
  std::vector<Item> items;
  for (int i : idx) {
    const ptycho_problem& q = probs[i];
    ptycho_plan pl = q.plan;
    const ptycho_params& p = pl->p;
    auto tag = [&](int rc) {
      g_last_error = "problem " + std::to_string(i) + ": " + g_last_error;
      return rc;
    };
    int rc;
    if ((rc = check_array(q.probe, "probe", true)) || (rc = check_array(q.obj, "obj", true)) ||
        (rc = check_array(q.meas_I, "meas_I", true)) || (!step && (rc = check_array(q.grad_obj, "grad_obj", false))) ||
        (!step && (rc = check_array(q.grad_probe, "grad_probe", false))))
      return tag(rc);
    if ((rc = check_positions(pl, q.pos_yx, st))) return tag(rc);
    float2 *gO = reinterpret_cast<float2*>(q.grad_obj), *gP = reinterpret_cast<float2*>(q.grad_probe);
    if (step) {
      const size_t nO = (size_t)p.S * p.H * p.W, nP = (size_t)p.M * p.M;
      if (!pl->g_obj && (rc = dev_alloc(&pl->g_obj, nO, "step object gradient"))) return tag(rc);
      if (!pl->g_probe && (rc = dev_alloc(&pl->g_probe, nP, "step probe gradient"))) return tag(rc);
      gO = pl->g_obj;
      gP = pl->g_probe;
    }
    items.push_back({i, pl, gO, gP});
  }
  for (int M : {64, 128}) {
    std::vector<Item> grp;
    for (const Item& it : items)
      if (it.pl->p.M == M) grp.push_back(it);
    for (int r = 0;; ++r) {
      std::vector<const Item*> live;
      for (const Item& it : grp)
        if ((int64_t)r * it.pl->chunk < it.pl->p.N) live.push_back(&it);
      if (live.empty()) break;
      for (size_t k0 = 0; k0 < live.size(); k0 += kMultiChainMax) {
        const size_t k1 = std::min(live.size(), k0 + (size_t)kMultiChainMax);
        MultiChainArgs m{};
        m.n = (int)(k1 - k0);
        for (size_t k = k0; k < k1; ++k) {
          const Item& it = *live[k];
          const ptycho_problem& q = probs[it.i];
          const int c0 = r * it.pl->chunk, n = std::min(it.pl->chunk, it.pl->p.N - c0);
          ChainArgs a = base_args(it.pl, q.pos_yx, q.probe, q.obj, q.meas_I);
          a.pos_begin = c0;
          a.n_pos = n;
          m.a[k - k0] = a;
          m.start[k - k0 + 1] = m.start[k - k0] + n;
          it.pl->tm.chain_positions += n;
        }
        ptycho_plan pl = live[k0]->pl;  // the launch is counted (and timed) on its first problem's plan
        TIMED(K_CHAIN, 1, launch_chain_multi(M, m, st));
      }
      for (const Item* it : live) {
        ptycho_plan pl = it->pl;
        const ptycho_problem& q = probs[it->i];
        const int c0 = r * pl->chunk, n = std::min(pl->chunk, pl->p.N - c0);
        if (it->gO) {
          // the single call's split: full chain waves, then the partial last wave
          const int tail = (pl->side && pl->wave > 0 && n > pl->wave) ? n % pl->wave : 0;
          int rc;
          if ((rc = accum_part(pl, q.pos_yx, q.probe, it->gO, c0, 0, n - tail, r > 0, st))) return rc;
          if (tail && (rc = accum_part(pl, q.pos_yx, q.probe, it->gO, c0, n - tail, tail, 1, st))) return rc;
        }
        if (it->gP)
          TIMED(K_PROBE, 2, launch_probe_grad(pl->ws_gp, n, pl->p.M, pl->gp_part, kProbeSplit, it->gP, r > 0, st));
        TIMED(K_OTHER, 1, launch_loss_accum(pl->loss_part, n, pl->d_scal, r > 0, st));
      }
    }
  }
  for (const Item& it : items) {
    ptycho_plan pl = it.pl;
    const ptycho_problem& q = probs[it.i];
    int rc;
    if ((rc = deliver_loss(pl, 0, q.loss_out, st))) return rc;
    if (step) {
      const ptycho_params& p = pl->p;
      TIMED(K_OTHER, 1, launch_axpy(reinterpret_cast<float2*>(q.obj), pl->g_obj, reinterpret_cast<float2*>(q.obj),
                                    -a_o, (size_t)p.S * p.H * p.W, st));
      TIMED(K_OTHER, 1, launch_axpy(reinterpret_cast<float2*>(q.probe), pl->g_probe,
                                    reinterpret_cast<float2*>(q.probe), -a_p, (size_t)p.M * p.M, st));
    }
  }
  return PTYCHO_OK;
}

// ptycho_loss_grad_host: host arrays in and out.  The inputs are staged in
// plan-owned device buffers; the intensities of all but the first chain wave
// go up on the copy stream while that wave runs.
int loss_grad_host_impl(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe, const ptycho_c64* obj,
                        const float* meas_I, double* loss_out, ptycho_c64* grad_obj, ptycho_c64* grad_probe,
                        cudaStream_t st) {
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  ptycho_plan pl = plan;
  const ptycho_params& p = pl->p;
  struct Arg {
    const void* ptr;
    const char* name;
    bool required;
  } args[] = {{pos_yx, "pos_yx", p.N > 0}, {probe, "probe", true},           {obj, "obj", true},
              {meas_I, "meas_I", p.N > 0}, {loss_out, "loss_out", true},      {grad_obj, "grad_obj", false},
              {grad_probe, "grad_probe", false}};
  for (const Arg& x : args) {
    if (!x.ptr) {
      if (x.required) return fail(PTYCHO_ERR_ARG, std::string(x.name) + " is NULL");
      continue;
    }
    if (is_device_ptr(x.ptr)) return fail(PTYCHO_ERR_ARG, std::string(x.name) + " must be a host pointer");
  }
  int rc;
  if (p.N > 0 && (rc = check_windows(p, pos_yx))) return rc;

  const size_t MM = (size_t)p.M * p.M, nO = (size_t)p.S * p.H * p.W;
  if (!pl->x_probe) {
    rc = PTYCHO_OK;
    if (!rc) rc = dev_alloc(&pl->x_pos, 2 * (size_t)p.N, "staged positions");
    if (!rc) rc = dev_alloc(&pl->x_probe, MM, "staged probe");
    if (!rc) rc = dev_alloc(&pl->x_obj, nO, "staged object");
    if (!rc) rc = dev_alloc(&pl->x_meas, (size_t)p.N * MM, "staged intensities");
    if (!rc) rc = dev_alloc(&pl->x_gO, nO, "staged object gradient");
    if (!rc) rc = dev_alloc(&pl->x_gP, MM, "staged probe gradient");
    cudaError_t e;
    if (!rc && ((e = cudaStreamCreateWithFlags(&pl->copy, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&pl->ev_first, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&pl->ev_rest, cudaEventDisableTiming)) != cudaSuccess))
      rc = cuda_fail(e, "copy stream");
    if (rc) {  // leave nothing half-made: the next call starts over
      cudaFree(pl->x_pos); cudaFree(pl->x_probe); cudaFree(pl->x_obj);
      cudaFree(pl->x_meas); cudaFree(pl->x_gO); cudaFree(pl->x_gP);
      pl->x_pos = nullptr; pl->x_probe = pl->x_obj = pl->x_gO = pl->x_gP = nullptr; pl->x_meas = nullptr;
      if (pl->ev_first) cudaEventDestroy(pl->ev_first);
      if (pl->ev_rest) cudaEventDestroy(pl->ev_rest);
      if (pl->copy) cudaStreamDestroy(pl->copy);
      pl->ev_first = pl->ev_rest = nullptr;
      pl->copy = nullptr;
      return rc;
    }
  }
  // Uploads in the order the chain needs them.  The copy stream starts after
  // the first part is up, so the two parts do not share the link, and after
  // everything earlier on st (a previous call still reading the buffers).
  const int n_first = pl->wave > 0 && pl->wave < p.N ? pl->wave : p.N;
  if (p.N > 0)
    CUDA_TRY(cudaMemcpyAsync(pl->x_pos, pos_yx, sizeof(int32_t) * 2 * (size_t)p.N, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(pl->x_probe, probe, sizeof(float2) * MM, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(pl->x_obj, obj, sizeof(float2) * nO, cudaMemcpyHostToDevice, st));
  if (p.N > 0)
    CUDA_TRY(cudaMemcpyAsync(pl->x_meas, meas_I, sizeof(float) * MM * (size_t)n_first, cudaMemcpyHostToDevice, st));
  cudaEvent_t rest = nullptr;
  if (n_first < p.N) {
    CUDA_TRY(cudaEventRecord(pl->ev_first, st));
    CUDA_TRY(cudaStreamWaitEvent(pl->copy, pl->ev_first, 0));
    CUDA_TRY(cudaMemcpyAsync(pl->x_meas + MM * (size_t)n_first, meas_I + MM * (size_t)n_first,
                             sizeof(float) * MM * (size_t)(p.N - n_first), cudaMemcpyHostToDevice, pl->copy));
    CUDA_TRY(cudaEventRecord(pl->ev_rest, pl->copy));
    rest = pl->ev_rest;
  }
  rc = run_loss_grad(pl, pl->x_pos, reinterpret_cast<const ptycho_c64*>(pl->x_probe),
                     reinterpret_cast<const ptycho_c64*>(pl->x_obj), pl->x_meas, grad_obj ? pl->x_gO : nullptr,
                     grad_probe ? pl->x_gP : nullptr, 0, nullptr, 0.f, nullptr, 0.f, st, n_first, rest);
  if (rc) {
    cudaStreamSynchronize(pl->copy);  // no upload left running into the buffers
    return rc;
  }
  if (grad_obj) CUDA_TRY(cudaMemcpyAsync(grad_obj, pl->x_gO, sizeof(float2) * nO, cudaMemcpyDeviceToHost, st));
  if (grad_probe) CUDA_TRY(cudaMemcpyAsync(grad_probe, pl->x_gP, sizeof(float2) * MM, cudaMemcpyDeviceToHost, st));
  // The call is synchronous, so it reports the device error word itself.
  CUDA_TRY(cudaMemcpyAsync(pl->h_flag, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if ((rc = deliver_loss(pl, 0, loss_out, st))) return rc;  // synchronises st
  if (const int h = *pl->h_flag) {
    CUDA_TRY(cudaMemsetAsync(pl->d_status, 0, sizeof(int), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return status_fail(h);
  }
  return PTYCHO_OK;
}

}  // namespace

extern "C" {

int ptycho_loss_grad_host(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe, const ptycho_c64* obj,
                          const float* meas_I, double* loss_out, ptycho_c64* grad_obj, ptycho_c64* grad_probe,
                          void* stream) {
  g_last_error.clear();
  return loss_grad_host_impl(plan, pos_yx, probe, obj, meas_I, loss_out, grad_obj, grad_probe,
                             static_cast<cudaStream_t>(stream));
}

int ptycho_loss_grad(ptycho_plan plan, const int32_t* pos_yx, const ptycho_c64* probe, const ptycho_c64* obj,
                     const float* meas_I, double* loss_out, ptycho_c64* grad_obj, ptycho_c64* grad_probe,
                     void* stream) {
  g_last_error.clear();
  return loss_grad_impl(plan, pos_yx, probe, obj, meas_I, loss_out, grad_obj, grad_probe,
                        static_cast<cudaStream_t>(stream));
}

int ptycho_step(ptycho_plan plan, const int32_t* pos_yx, ptycho_c64* probe, ptycho_c64* obj, const float* meas_I,
                double alpha_obj, double alpha_probe, int32_t line_search, double* loss_out, double* t_out,
                void* stream) {
  g_last_error.clear();
  return step_impl(plan, pos_yx, probe, obj, meas_I, alpha_obj, alpha_probe, line_search, loss_out, t_out,
                   static_cast<cudaStream_t>(stream));
}

int ptycho_step_accumulate(ptycho_plan plan, const int32_t* pos_yx, ptycho_c64* probe, ptycho_c64* obj,
                           const float* meas_I, double alpha_obj, double alpha_probe, ptycho_c64* acc,
                           int32_t flush, double* loss_out, void* stream) {
  g_last_error.clear();
  if (!plan) return fail(PTYCHO_ERR_ARG, "plan is NULL");
  int rc;
  if ((rc = check_array(acc, "acc", true))) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((rc = step_impl(plan, pos_yx, probe, obj, meas_I, alpha_obj, alpha_probe, 0, loss_out, nullptr, st)))
    return rc;
  // step_impl left this call's object gradient in the plan's step buffer
  const ptycho_params& p = plan->p;
  const size_t nO = (size_t)p.S * p.H * p.W;
  float2* A = reinterpret_cast<float2*>(acc);
  float2* O = reinterpret_cast<float2*>(obj);
  ptycho_plan pl = plan;
  TIMED_ON(st, K_OTHER, 1, launch_axpy(A, plan->g_obj, A, 1.0, nO, st));  // AccBuf += dF/dO
  if (flush) {
    TIMED_ON(st, K_OTHER, 1, launch_axpy(O, A, O, -alpha_obj, nO, st));  // second update
    CUDA_TRY(cudaMemsetAsync(A, 0, nO * sizeof(float2), st));
  }
  return PTYCHO_OK;
}

int ptycho_multi_loss_grad(const ptycho_problem* problems, int32_t n, void* stream) {
  g_last_error.clear();
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int> fused;
  int rc = run_multi(problems, n, [&](const ptycho_problem& q) {
    if (fusable(q.plan) && (q.grad_obj || q.grad_probe)) {  // loss-only problems take the cheaper chain
      fused.push_back((int)(&q - problems));
      return PTYCHO_OK;
    }
    return loss_grad_impl(q.plan, q.pos_yx, q.probe, q.obj, q.meas_I, q.loss_out, q.grad_obj, q.grad_probe, st);
  });
  return rc ? rc : run_multi_fused(problems, fused, false, 0.0, 0.0, st);
}

int ptycho_multi_step(const ptycho_problem* problems, int32_t n, double alpha_obj, double alpha_probe,
                      void* stream) {
  g_last_error.clear();
  if (!std::isfinite(alpha_obj) || !std::isfinite(alpha_probe))
    return fail(PTYCHO_ERR_ARG, "step sizes must be finite");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int> fused;
  int rc = run_multi(problems, n, [&](const ptycho_problem& q) {
    if (fusable(q.plan)) {
      fused.push_back((int)(&q - problems));
      return PTYCHO_OK;
    }
    return step_impl(q.plan, q.pos_yx, q.probe, q.obj, q.meas_I, alpha_obj, alpha_probe, 0, q.loss_out, nullptr,
                     st);
  });
  return rc ? rc : run_multi_fused(problems, fused, true, alpha_obj, alpha_probe, st);
}

int ptycho_potential_to_transmission(const float* V, ptycho_c64* obj, int64_t n, double sigma, void* stream) {
  g_last_error.clear();
  if (n < 0 || !std::isfinite(sigma)) return fail(PTYCHO_ERR_ARG, "n must be >= 0 and sigma finite");
  if (n == 0) return PTYCHO_OK;
  int rc;
  if ((rc = check_array(obj, "obj", true))) return rc;
  if (!is_device_ptr(V) || !aligned(V, 4)) return fail(PTYCHO_ERR_ARG, "V must be a 4-byte aligned device pointer");
  CUDA_TRY(launch_potential_to_transmission(V, reinterpret_cast<float2*>(obj), sigma, (size_t)n,
                                            static_cast<cudaStream_t>(stream)));
  return PTYCHO_OK;
}

int ptycho_potential_grad(const ptycho_c64* obj, const ptycho_c64* grad_obj, float* grad_V, int64_t n,
                          double sigma, void* stream) {
  g_last_error.clear();
  if (n < 0 || !std::isfinite(sigma)) return fail(PTYCHO_ERR_ARG, "n must be >= 0 and sigma finite");
  if (n == 0) return PTYCHO_OK;
  int rc;
  if ((rc = check_array(obj, "obj", true)) || (rc = check_array(grad_obj, "grad_obj", true))) return rc;
  if (!is_device_ptr(grad_V) || !aligned(grad_V, 4))
    return fail(PTYCHO_ERR_ARG, "grad_V must be a 4-byte aligned device pointer");
  CUDA_TRY(launch_potential_grad(reinterpret_cast<const float2*>(obj), reinterpret_cast<const float2*>(grad_obj),
                                 grad_V, sigma, (size_t)n, static_cast<cudaStream_t>(stream)));
  return PTYCHO_OK;
}

}  // extern "C"
