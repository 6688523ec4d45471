// Adjoint operator without any device allocation (lps_adjoint_noalloc in lps_api.h).
//
// Some callers cannot allocate device memory at the point where they need the operator:
// code that runs while another component owns the device memory pool (a framework's caching
// allocator, a scanner pipeline that reserves all memory up front), real-time loops that
// forbid allocation after start-up, and callers that must not synchronise the device (a
// cudaMalloc/cudaFree can). For them this entry point runs the same kernels as lps_adjoint
// with the scratch they need (line table, twiddles and the samples moved to hybrid space)
// in one file-scope device array of fixed size, LPS_NOALLOC_SCRATCH_BYTES.
//
// The array is part of the library image: every GPU that loads the library holds it until
// the process exits. All calls share it and it keeps the last call's contents, so calls
// whose work overlaps on the GPU (different streams, or different host threads) race on it;
// callers must order such calls. Everything a call reads from the array is written by that
// call first. Calls queued back to back on one stream need no host synchronisation between
// them: the tables are uploaded with cudaMemcpyAsync from pageable host memory, which returns
// only once the source has been consumed, so the next call may rewrite the host staging
// buffers, and its device writes are ordered after the previous call's kernels.
#include "lps_api.h"
#include "lps_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace lps {
int make_geom(const lps_params* p, Geom* g);
void set_err(const char* fmt, ...);
}

using namespace lps;

static __device__ __align__(256) unsigned char g_noalloc_scratch[LPS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_dev_scratch[kMaxDevices] = {};   // device address of the array, per device
int g_lines[1024 * LPS_MAX_NC];                     // host staging of the line table (static)
float2 g_tw[3 * 1024];                              // host staging of the twiddles (static)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Memory kind of a pointer under unified addressing: 1 device (or managed), 0 host, -1 the
// query failed. cudaPointerGetAttributes allocates nothing.
int pointer_kind(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

}  // namespace

extern "C" int lps_adjoint_noalloc(int nx, int ny, int nz, int ncoil, int fft_z, const uint8_t* mask,
                                   const void* coils, const void* kdata, int nlines, void* image, void* stream) {
  if (!mask || !coils || !kdata || !image) {
    set_err("lps_adjoint_noalloc: mask, coils, kdata and image must be non-NULL");
    return LPS_ERR_INVALID_ARG;
  }
  // The kernels read coils and kdata and write image directly, and the host reads the mask:
  // anything else is refused here, before any copy or launch.
  if (pointer_kind(coils) != 1 || pointer_kind(kdata) != 1 || pointer_kind(image) != 1) {
    set_err("lps_adjoint_noalloc: coils, kdata and image must be device memory");
    return LPS_ERR_INVALID_ARG;
  }
  if (pointer_kind(mask) == 1) {
    set_err("lps_adjoint_noalloc: mask must be host memory");
    return LPS_ERR_INVALID_ARG;
  }
  lps_params p;
  lps_params_init(&p);
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.ncoil = ncoil;
  p.fft_z = fft_z;
  Geom g;
  int rc = make_geom(&p, &g);
  if (rc) return rc;
  int m = 0;
  for (int i = 0; i < ny * nz; ++i) m += mask[i] != 0;
  if (m == 0) {
    set_err("lps_adjoint_noalloc: mask has no sampled entry");
    return LPS_ERR_INVALID_ARG;
  }
  if (m != nlines) {
    set_err("lps_adjoint_noalloc: nlines %d != %d set mask entries", nlines, m);
    return LPS_ERR_INVALID_ARG;
  }
  const int mpad = (m + 1) & ~1;
  g.mpad = mpad;
  // scratch layout: [persist][tw_x][tw_y][tw_z][lines][hybrid samples]
  const size_t o_persist = 0;
  const size_t o_tx = o_persist + align256(sizeof(DevPersist));
  const size_t o_ty = o_tx + align256((size_t)nx * sizeof(float2));
  const size_t o_tz = o_ty + align256((size_t)ny * sizeof(float2));
  const size_t o_lines = o_tz + align256((size_t)nz * sizeof(float2));
  const size_t o_hyb = o_lines + align256((size_t)ny * nz * sizeof(int));
  const size_t need = o_hyb + ((size_t)nx * ncoil * mpad + 4) * sizeof(float2);
  if (need > LPS_NOALLOC_SCRATCH_BYTES) {   // beyond the fixed scratch
    set_err("lps_adjoint_noalloc: needs %zu bytes of scratch > LPS_NOALLOC_SCRATCH_BYTES (%u)", need,
            (unsigned)LPS_NOALLOC_SCRATCH_BYTES);
    return LPS_ERR_UNSUPPORTED;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err("lps_adjoint_noalloc: no current device (or device index >= %d)", kMaxDevices);
    return LPS_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_dev_scratch[dev]) {
    // once per device, with that device current: the device address of the array
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_err("lps_adjoint_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return LPS_ERR_CUDA;
    }
    g_dev_scratch[dev] = static_cast<unsigned char*>(ptr);
  }
  unsigned char* base = g_dev_scratch[dev];
  DevPersist* persist = reinterpret_cast<DevPersist*>(base + o_persist);
  float2* tw_x = reinterpret_cast<float2*>(base + o_tx);
  float2* tw_y = reinterpret_cast<float2*>(base + o_ty);
  float2* tw_z = reinterpret_cast<float2*>(base + o_tz);
  int* lines = reinterpret_cast<int*>(base + o_lines);
  float2* hyb = reinterpret_cast<float2*>(base + o_hyb);

  // host-side tables (static staging buffers, copied before the call returns)
  int k = 0;
  for (int a = 0; a < nz; ++a)
    for (int ky = 0; ky < ny; ++ky)
      if (mask[(size_t)a * ny + ky]) g_lines[k++] = a * g.nyp + ky;
  auto fill_tw = [](float2* t, int n) {
    for (int q = 0; q < n; ++q) {
      const double ang = 2.0 * M_PI * (double)q / (double)n;
      t[q] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
    }
  };
  fill_tw(g_tw, nx);
  fill_tw(g_tw + nx, ny);
  fill_tw(g_tw + nx + ny, nz);
  DevPersist hp;
  std::memset(&hp, 0, sizeof(hp));
  hp.nlines = m;
  // copies from pageable host memory return once the source has been read, so the static
  // staging buffers may be rewritten by the next call
  if (cudaMemcpyAsync(persist, &hp, sizeof(hp), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(tw_x, g_tw, (size_t)nx * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(tw_y, g_tw + nx, (size_t)ny * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(tw_z, g_tw + nx + ny, (size_t)nz * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(lines, g_lines, (size_t)m * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_err("lps_adjoint_noalloc: table upload failed: %s", cudaGetErrorString(cudaGetLastError()));
    return LPS_ERR_CUDA;
  }

  XfftArgs x{};
  x.g = g;
  x.in = static_cast<const float2*>(kdata);
  x.out = hyb;
  x.tw_x = tw_x;
  x.persist = persist;
  x.inverse = 1;
  cudaError_t le = launch_xfft(x, st);
  if (le != cudaSuccess) {
    set_err("lps_adjoint_noalloc: kx transform launch failed: %s", cudaGetErrorString(le));
    return LPS_ERR_CUDA;
  }
  DcArgs d{};
  d.g = g;
  d.coils = static_cast<const float2*>(coils);
  d.dhyb = hyb;
  d.lines = lines;
  d.tw_y = tw_y;
  d.tw_z = tw_z;
  d.persist = persist;
  d.X = static_cast<float2*>(image);
  le = launch_dc(d, kDcAdjoint, st);
  if (le != cudaSuccess) {
    set_err("lps_adjoint_noalloc: adjoint launch failed: %s", cudaGetErrorString(le));
    return LPS_ERR_CUDA;
  }
  return LPS_OK;
}
