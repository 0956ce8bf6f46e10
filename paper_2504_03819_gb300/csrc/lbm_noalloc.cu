// lbm_step_noalloc: one time step for callers that cannot allocate device
// memory.  The step's scratch fields live in a file-scope static device array
// instead of a caller-provided workspace; the kernels are the same ones
// lbm_step launches (FP32 storage, populations exchanged unshifted).
#include <mutex>

#include "lbm_internal.h"

namespace {

// Scratch layout for N <= LBM_NOALLOC_MAX_NODES nodes, mirroring the field
// part of the workspace: 20 floats per node (rho, j, mu', u, F, phi, Q, shift
// bases, mu0), the boundary list (one int per node), the solid-neighbour bitmasks
// and inverse fluid-weight sums (one word each per node), the compaction
// counts (one int per 256 nodes) and two status ints.
constexpr size_t kMax = LBM_NOALLOC_MAX_NODES;
constexpr size_t kFieldBytes = 20 * kMax * sizeof(float);
constexpr size_t kBndOff = kFieldBytes;
constexpr size_t kNbrOff = kBndOff + kMax * sizeof(int);
constexpr size_t kInvDenOff = kNbrOff + kMax * sizeof(uint32_t);
constexpr size_t kScanOff = kInvDenOff + kMax * sizeof(float);
constexpr size_t kStatusOff = kScanOff + (kMax / 256 + 2) * sizeof(int);
constexpr size_t kScratchBytes = kStatusOff + 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host code cannot use g_noalloc_scratch as a device address: its device
// address is looked up once per device with cudaGetSymbolAddress.  The cached
// address belongs to the device's primary context; it does not survive
// cudaDeviceReset (or any other teardown of that context) in this process.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices];

int scratch_for_current_device(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_step_noalloc(const float *f_in, float *f_out, const uint8_t *solid_mask, int nx, int ny,
                                int nz, const lbm_params *params, void *cuda_stream) {
  if (!f_in || !f_out || !params || (const void *)f_in == (const void *)f_out) return LBM_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
  const long long N = (long long)nx * ny * nz;
  if (N > (long long)kMax) return LBM_ERR_SIZE;
  void *base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != LBM_OK) return rc;

  lbm_ctx ctx{};  // host-side only; views into the static scratch and the caller's buffers
  ctx.nx = nx;
  ctx.ny = ny;
  ctx.nz = nz;
  ctx.N = (int)N;
  ctx.storage = LBM_F32;
  ctx.stream = (cudaStream_t)cuda_stream;
  ctx.mask = solid_mask;
  ctx.f[0] = const_cast<float *>(f_in);  // read only: the step writes f[1 - cur]
  ctx.f[1] = f_out;
  ctx.cur = 0;
  float *fl = (float *)base;
  const size_t n = (size_t)N;
  ctx.fld.rho = fl;
  ctx.fld.j = fl + n;
  ctx.fld.mu = fl + 4 * n;
  ctx.fld.u = fl + 5 * n;
  ctx.fld.F = fl + 8 * n;
  ctx.fld.phi = fl + 11 * n;
  ctx.fld.Q = fl + 14 * n;
  ctx.fld.sb = fl + 17 * n;
  ctx.fld.mu0 = fl + 19 * n;
  // one step: the moments of its output are not produced (one moment set)
  ctx.mom[0] = ctx.mom[1] = lbm::Moments{ctx.fld.rho, ctx.fld.j, ctx.fld.mu0};
  ctx.no_mom = 1;
  ctx.bnd = (int *)((char *)base + kBndOff);
  ctx.nbr = (uint32_t *)((char *)base + kNbrOff);
  ctx.inv_den = (float *)((char *)base + kInvDenOff);
  ctx.scan = (int *)((char *)base + kScanOff);
  ctx.red_partial = nullptr;
  ctx.status = (int *)((char *)base + kStatusOff);
  ctx.kp.nx = nx;
  ctx.kp.ny = ny;
  ctx.kp.nz = nz;
  ctx.kp.N = (int)N;

  // populations cross this entry point unshifted: constant shift rho_0 = 0
  lbm_params p = *params;
  p.shift_mode = LBM_SHIFT_CONST;
  p.rho_shift = 0.0;
  rc = lbm_set_params(&ctx, &p);
  if (rc != LBM_OK) return rc;

  cudaGetLastError();
  // the array keeps the previous call's contents: clear what must start at 0
  cudaMemsetAsync(base, 0, 20 * n * sizeof(float), ctx.stream);
  cudaMemsetAsync(ctx.status, 0, 2 * sizeof(int), ctx.stream);
  cudaMemsetAsync(f_out, 0, 27 * n * sizeof(float), ctx.stream);  // solid-node slots stay 0
  if (solid_mask) {
    lbm::launch_mark_boundary(&ctx);
    int cnt = 0;
    cudaMemcpyAsync(&cnt, ctx.status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream);
    if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) {
      cudaGetLastError();
      return LBM_ERR_CUDA;
    }
    ctx.n_bnd = cnt;
  }
  ctx.have_state = 1;
  lbm::launch_step(&ctx);
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  // the step's status word lives in the shared array: read it before the
  // next call can clear it (a copy into a host int, no allocation)
  int st = 0;
  if (cudaMemcpyAsync(&st, ctx.status, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx.stream) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  if (st & lbm::STATUS_NONFINITE) return LBM_ERR_NONFINITE;
  if (st & lbm::STATUS_DOMAIN) return LBM_ERR_DOMAIN;
  if (st & lbm::STATUS_TIMEOUT) return LBM_ERR_TIMEOUT;
  return LBM_OK;
}
