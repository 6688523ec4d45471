// Transform of the sampled k-space lines along the fully sampled readout axis kx
// (acquisition operator of Sec. 2). Because the line mask does not depend on kx, the
// orthonormal x-DFT is applied once per frame to move the samples to the hybrid
// (x, ky, kz) space, where the data-consistency step works plane by plane:
//   inverse: k-space [coil][line][kx] -> hybrid [x][coil][line]   (d' = F_x^H d)
//   forward: hybrid [x][coil][line]   -> k-space [coil][line][kx] (d = F_x h)
// One CTA transforms kLines lines of one coil; the transpose goes through shared memory
// so that both the row reads and the x-major writes are contiguous.
#include "lps_internal.cuh"

namespace lps {

constexpr int kLines = 16;

// A plan that holds a slab of the volume (planes x0 .. x0+nx-1 of nxt) transforms whole
// readouts of nxt samples; the inverse keeps its own planes, the forward takes the planes it
// does not hold as zero (its output is the slab's share of E x, which the slabs add up).
__global__ void __launch_bounds__(kThreads) k_xfft(const XfftArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom& g = a.g;
  const int nx = g.nxt, nxp = nx + 1, x0 = g.x0, nxl = g.nx;
  float2* bufA = reinterpret_cast<float2*>(smem);
  float2* bufB = bufA + kLines * nxp;
  float2* tw = bufB + kLines * nxp;
  const int m = a.persist->nlines;
  const int c = blockIdx.y;
  const int l0 = blockIdx.x * kLines;
  if (l0 >= m) return;
  const int nl = min(kLines, m - l0);
  const int tid = threadIdx.x;
  for (int i = tid; i < nx; i += kThreads) tw[i] = a.tw_x[i];
  const int tot = kLines * nx;
  if (a.inverse) {
    const float2* src = a.in + ((long long)c * m + l0) * nx;
    for (int e = tid; e < tot; e += kThreads) {
      const int l = e / nx, k = e - (e / nx) * nx;
      bufA[l * nxp + k] = (l < nl) ? src[(long long)l * nx + k] : make_float2(0.f, 0.f);
    }
  } else {
    for (int e = tid; e < tot; e += kThreads) {
      const int x = e / kLines, l = e - (e / kLines) * kLines;
      const int xl = x - x0;
      bufA[l * nxp + x] = (l < nl && xl >= 0 && xl < nxl) ? a.in[((long long)xl * g.ncoil + c) * g.mpad + l0 + l]
                                                          : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  float2* s = bufA;
  float2* d = bufB;
  fft_run(&s, &d, g.px, kLines, 1, nxp, tw, a.inverse != 0);
  const float sc = g.scale_x;
  if (a.inverse) {
    for (int e = tid; e < kLines * nxl; e += kThreads) {
      const int xl = e / kLines, l = e - (e / kLines) * kLines;
      if (l < nl) a.out[((long long)xl * g.ncoil + c) * g.mpad + l0 + l] = cscale(s[l * nxp + x0 + xl], sc);
    }
  } else {
    float2* dst = a.out + ((long long)c * m + l0) * nx;
    for (int e = tid; e < tot; e += kThreads) {
      const int l = e / nx, k = e - (e / nx) * nx;
      if (l < nl) dst[(long long)l * nx + k] = cscale(s[l * nxp + k], sc);
    }
  }
}

size_t xfft_smem_bytes(const Geom& g) {
  return (size_t)(2 * kLines * (g.nxt + 1) + g.nxt) * sizeof(float2);
}

// Grid: (ceil(nlines_cap / kLines), ncoil); CTAs past the current line count exit.
cudaError_t launch_xfft(const XfftArgs& a, cudaStream_t st) {
  const size_t smem = xfft_smem_bytes(a.g);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_xfft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int cap = a.g.mpad;
  dim3 grid((cap + kLines - 1) / kLines, a.g.ncoil);
  k_xfft<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lps
