// Multi-vector product of a stored float32 dense operator on the tensor cores
// with no device allocation: every temporary lives in one fixed device array.
//
// The operation is the same y = X x as cal_matvec's tensor-core branch (real
// embedding of the complex vectors, 3xTF32 GEMM, unembedding); only the
// scratch differs. The array holds, at 256-byte aligned offsets:
//   Bt  [NB][2 cols] float   embedded right-hand sides (fully rewritten per call)
//   Z   [rows][NB]   float   GEMM output (zeroed per call by the GEMM launcher:
//                            split-K partial sums are added into it)
//   err int                  bounded-wait flag (zeroed per call)
//   xp  [nrhs+1][cols] float2  odd nrhs only: vectors padded with one zero vector
//                            (the padding vector is zeroed per call)
// Every call on a device shares the one array, so calls whose GPU work
// overlaps (two streams, or two host threads) race on it; callers serialise.
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "solve.h"

namespace cal {
namespace {

constexpr size_t kScratchBytes = CAL_MATVEC_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_base[kMaxDevices] = {};

// Device address of g_scratch on `device`, looked up on the first call on that
// device with the device current (the caller has made it current) and kept for
// the life of the process: a cudaDeviceReset of that device would leave the
// kept address stale, so the library is not to be used across one.
int scratch_base(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return fail(CAL_EINVAL, "static scratch: device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_base[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(CAL_ECUDA, "static scratch: cudaGetSymbolAddress failed (%s)", cudaGetErrorString(e));
    g_scratch_base[device] = p;
  }
  *out = (unsigned char*)g_scratch_base[device];
  return CAL_OK;
}

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// y[j][r] = Z[r][2j] + i Z[r][2j+1], j < ncol
__global__ void unembed_static_kernel(const float* __restrict__ Z, int64_t rows, int NB, int ncol,
                                      float2* __restrict__ y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r < rows && j < ncol) y[(int64_t)j * rows + r] = make_float2(Z[r * NB + 2 * j], Z[r * NB + 2 * j + 1]);
}

}  // namespace
}  // namespace cal

using namespace cal;

extern "C" int cal_matvec_static(const cal_op* op, int which, const void* x, void* y, int64_t nrhs, void* stream) {
  if (!op || !x || !y) return fail(CAL_EINVAL, "cal_matvec_static: NULL argument");
  const Op& o = op->impl;
  const void* X = which == CAL_OP_S ? o.d_S : (which == CAL_OP_C ? o.d_C : nullptr);
  if (!X) return fail(CAL_EINVAL, "cal_matvec_static: operator %d was not assembled", which);
  if (o.precision != CAL_FP32 || o.format != CAL_DENSE)
    return fail(CAL_EINVAL, "cal_matvec_static: needs a float32 dense operator");
  if (nrhs < 1 || nrhs > CAL_MATVEC_STATIC_MAX_NRHS)
    return fail(CAL_EINVAL, "cal_matvec_static: nrhs = %lld outside [1, %d]", (long long)nrhs,
                CAL_MATVEC_STATIC_MAX_NRHS);
  if (o.cols % 2) return fail(CAL_EINVAL, "cal_matvec_static: the operator needs an even column count");
  const int64_t rows = o.rows, cols = o.cols;
  const int n = (int)nrhs;
  const int npair = (n + 1) / 2;
  const int NB = ((4 * npair + 15) / 16) * 16;
  const size_t b_Bt = round256((size_t)NB * 2 * cols * sizeof(float));
  const size_t b_Z = round256((size_t)rows * NB * sizeof(float));
  const size_t b_err = 256;
  const size_t b_xp = (n % 2) ? round256((size_t)(n + 1) * cols * sizeof(float2)) : 0;
  const size_t need = b_Bt + b_Z + b_err + b_xp;
  if (need > kScratchBytes)
    return fail(CAL_EINVAL,
                "cal_matvec_static: %lld x %lld operator with %d vectors needs %zu scratch bytes, above the "
                "fixed maximum of %zu",
                (long long)rows, (long long)cols, n, need, kScratchBytes);
  cudaPointerAttributes ax{}, ay{};
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ay, y) != cudaSuccess ||
      (ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged) ||
      (ay.type != cudaMemoryTypeDevice && ay.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail(CAL_EINVAL, "cal_matvec_static: x and y must be device pointers");
  }
  if ((ax.type == cudaMemoryTypeDevice && ax.device != o.ctx->device) ||
      (ay.type == cudaMemoryTypeDevice && ay.device != o.ctx->device))
    return fail(CAL_EINVAL, "cal_matvec_static: x and y must be on the operator's device %d", o.ctx->device);
  // the caller's current device is put back on every return path
  int prev_device = -1;
  CAL_TRY_CUDA(cudaGetDevice(&prev_device));
  struct Restore {
    int dev;
    ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
  } restore{prev_device};
  CAL_TRY_CUDA(cudaSetDevice(o.ctx->device));
  unsigned char* base;
  int rc = scratch_base(o.ctx->device, &base);
  if (rc) return rc;
  float* Bt = (float*)base;
  float* Z = (float*)(base + b_Bt);
  int* err = (int*)(base + b_Bt + b_Z);
  float2* xp = b_xp ? (float2*)(base + b_Bt + b_Z + b_err) : nullptr;
  cudaStream_t st = stream ? (cudaStream_t)stream : o.ctx->stream;
  CAL_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const float2* xin = (const float2*)x;
  if (xp) {  // pad to an even number of vectors with one zero vector
    CAL_TRY_CUDA(cudaMemcpyAsync(xp, x, (size_t)n * cols * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    CAL_TRY_CUDA(cudaMemsetAsync(xp + (size_t)n * cols, 0, (size_t)cols * sizeof(float2), st));
    xin = xp;
  }
  rc = embed_rhs<float2>(xin, npair, cols, 0, cols, Bt, NB, st);
  if (!rc) rc = gemm_tf32x3((const float*)X, rows, 2 * cols, Bt, NB, Z, err, o.ctx->n_sm, st);
  if (!rc) {
    unembed_static_kernel<<<dim3((unsigned)((rows + 255) / 256), n), 256, 0, st>>>(Z, rows, NB, n, (float2*)y);
    note_launch();
    CAL_TRY_CUDA(cudaGetLastError());
  }
  int herr = 0;
  CAL_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CAL_TRY_CUDA(cudaStreamSynchronize(st));
  if (!rc && herr) rc = fail(CAL_ETIMEOUT, "cal_matvec_static: a bounded wait of the tensor-core product gave up");
  return rc;
}
