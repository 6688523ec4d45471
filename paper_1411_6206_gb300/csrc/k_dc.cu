// Launchers of the data-consistency kernel k_dc (k_dc.cuh): runtime-sized Stockham variants
// (instantiated here) and the register-transform update (instantiated per nz in
// k_dc_rt_nz*.cu).
#include "k_dc.cuh"

#include <algorithm>

namespace lps {

int dc_ept(const Geom& g) { return dc_ept_of(g.plane); }

size_t dc_smem_bytes(const Geom& g) {
  size_t b = 0;
  b += 2 * (size_t)g.planeP * sizeof(float2);
  if (!g.dc_direct) b += 2 * (size_t)g.plane * sizeof(float2);   // staged coil planes
  b += (size_t)(g.ny + g.nz + ((g.ny + g.nz) & 1)) * sizeof(float2);
  b += 3 * sizeof(uint64_t);
  b += 32 * sizeof(float);
  b += (size_t)g.nz * g.nz * sizeof(float2);   // W of the iteration form
  return b;
}

template <int MODE, bool STAGE, bool HALF>
static cudaError_t launch_dc_m(const DcArgs& a, cudaStream_t st) {
  const size_t smem = dc_smem_bytes(a.g);
  switch (dc_ept(a.g)) {
    case 1: return launch_dc_t<1, MODE, STAGE, HALF>(a, smem, st);
    case 2: return launch_dc_t<2, MODE, STAGE, HALF>(a, smem, st);
    case 4: return launch_dc_t<4, MODE, STAGE, HALF>(a, smem, st);
    case 8: return launch_dc_t<8, MODE, STAGE, HALF>(a, smem, st);
    case 16: return launch_dc_t<16, MODE, STAGE, HALF>(a, smem, st);
    case 24: return launch_dc_t<24, MODE, STAGE, HALF>(a, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// Staged coil planes are copied in float32 (the rounded maps); the direct variant of the update
// reads the half-precision copy when the plan keeps one.
template <int MODE>
static cudaError_t launch_dc_s(const DcArgs& a, cudaStream_t st) {
  if (!a.g.dc_direct) return launch_dc_m<MODE, true, false>(a, st);
  if constexpr (MODE == kDcUpdate) {
    if (a.coils_h) return launch_dc_m<MODE, false, true>(a, st);
  }
  return launch_dc_m<MODE, false, false>(a, st);
}

cudaError_t launch_dc_fixed(const DcArgs& a, int mode, cudaStream_t st);

// Shared memory of the register-transform update: the direct kernel's layout with the W
// region replaced by the larger of itself and the transform loop's region.
static size_t dc_rt_smem_bytes(const Geom& g, int dsm_slots) {
  Geom gd = g;
  gd.dc_direct = 1;
  return dc_smem_bytes(gd) - (size_t)g.nz * g.nz * sizeof(float2) + rt_region_bytes(g.nz, g.ny, dsm_slots);
}

bool dc_rt_geometry(const Geom& g) {
  const int q = g.ny / 16;
  if (g.cs != 1 || g.ny % 16 != 0 || q < 4 || q > 10 || dc_has_fixed(g)) return false;
  switch (g.nz) {
    case 8: case 10: case 12: case 14: case 16: case 20: case 24: case 28: case 32: return true;
    default: return false;
  }
}

bool dc_rt_applies(const Geom& g) {
  return g.dc_rt && !g.dc_generic && dc_rt_geometry(g) && dc_rt_smem_bytes(g, 0) <= 227 * 1024;
}

// cudaErrorNotSupported where the plane has no register-transform instantiation (or the plan
// keeps half-precision coil maps, which the runtime-sized kernel reads).
static cudaError_t launch_dc_rt(const DcArgs& a, cudaStream_t st) {
  if (!dc_rt_applies(a.g) || a.coils_h) return cudaErrorNotSupported;
  // slots for a coil's samples in shared memory: the line capacity, or what is left of the
  // 227 KB (a frame with more lines reads them from L2)
  DcArgs b = a;
  const size_t fixed = dc_rt_smem_bytes(a.g, 0);
  b.g.dc_rt_dsm = (int)std::min<size_t>((size_t)a.g.mpad, (227 * 1024 - fixed) / sizeof(float2)) & ~1;
  const size_t smem = dc_rt_smem_bytes(b.g, b.g.dc_rt_dsm);
#define LPS_RT_DISPATCH(NZ) \
  case NZ: return launch_dc_rt_nz<NZ>(b, smem, st);
  switch (a.g.nz) {
    LPS_RT_NZ_LIST(LPS_RT_DISPATCH)
    default: return cudaErrorNotSupported;
  }
#undef LPS_RT_DISPATCH
}

// One persistent launch over a batch's descriptor table (operator form of the update): each CTA
// takes (member, plane) items from an atomic counter, copies the member's arguments to shared
// memory and runs the plane with the runtime-sized body (coil maps read from L2, up to 24
// elements per thread, the shared memory of the largest member). No CTA waits on another.
__global__ void __launch_bounds__(kThreads, 1) k_dc_persist(const DcArgs* __restrict__ table,
                                                          const int* __restrict__ start, int nm, int* counter) {
  __shared__ DcArgs sa;
  __shared__ int item_s, member_s;
  const int total = start[nm];
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
      int m = 0;
      while (m + 1 < nm && start[m + 1] <= it) ++m;
      item_s = it;
      member_s = m;
    }
    __syncthreads();
    const int it = item_s, m = member_s;
    if (it >= total) return;
    const int* src = reinterpret_cast<const int*>(table + m);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(DcArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    dc_plane<24, kDcUpdate, false, false, 0, 0>(sa, it - start[m]);
    __syncthreads();
  }
}
static_assert(sizeof(DcArgs) % sizeof(int) == 0, "DcArgs copied as words");

// The persistent form needs planes of at most 24 * kThreads elements; smem: the largest
// member's runtime-sized direct layout.
bool dc_persist_fits(const Geom& g) {
  Geom gd = g;
  gd.dc_direct = 1;
  return g.plane <= 24 * kThreads && dc_smem_bytes(gd) + sizeof(DcArgs) + 64 <= 227 * 1024;
}

size_t dc_persist_smem(const Geom& g) {
  Geom gd = g;
  gd.dc_direct = 1;
  return dc_smem_bytes(gd);
}

cudaError_t launch_dc_persist(const DcArgs* table, const int* start, int nm, int* counter, size_t smem,
                              cudaStream_t st) {
  // the kernel's static shared memory (its argument copy) counts against the same 227 KB
  cudaError_t e = cudaFuncSetAttribute(k_dc_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dc_persist, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_dc_persist<<<per_sm * sms, kThreads, smem, st>>>(table, start, nm, counter);
  return cudaGetLastError();
}

// The update of a 128 x 16 plane goes to the register-transform kernel (k_dc_reg) unless the
// plan selected another variant; planes of ny = 16 Q (Q = 4..10) by even nz <= 32 to k_dc with
// the register-transform coil loop; other plane sizes with a compile-time specialisation go to
// k_dc_fixed; the rest to k_dc.
cudaError_t launch_dc(const DcArgs& a, int mode, cudaStream_t st) {
  if (mode == kDcUpdate) {
    const cudaError_t er = launch_dc_reg(a, st);
    if (er != cudaErrorNotSupported) return er;
    const cudaError_t et = launch_dc_rt(a, st);
    if (et != cudaErrorNotSupported) return et;
  }
  const cudaError_t ef = launch_dc_fixed(a, mode, st);
  if (ef != cudaErrorNotSupported) return ef;
  if (dc_smem_bytes(a.g) > 227 * 1024) return cudaErrorInvalidValue;
  switch (mode) {
    case kDcUpdate: return launch_dc_s<kDcUpdate>(a, st);
    case kDcAdjoint: return launch_dc_s<kDcAdjoint>(a, st);
    case kDcForward: return launch_dc_s<kDcForward>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lps
