// Pressure map without any device allocation (tc_pressure_map_noalloc).
//
// Same computation as the env's pressure map -- per contact face the
// pressure p = -n.sigma.n of its parent tet on the deformed face and the
// face area, their area-weighted mean per contact vertex, and barycentric
// interpolation at every pixel -- but from caller-supplied device arrays, with
// the per-face and per-vertex intermediates in a file-scope device array
// instead of memory obtained from an allocator.  It serves callers that cannot
// allocate device memory at the point of the call (for example a real-time
// loop that forbids allocator calls after start-up, or code that runs inside
// someone else's memory pool), so it calls no cudaMalloc, cudaFree or
// allocating library routine.
#include <mutex>

#include "env.cuh"
#include "prof.cuh"

namespace tc {

// Capacity of the shared scratch: per-face pressure and area, per-vertex
// pressure.  Every GPU that loads the library holds this array until exit.
constexpr int kNoAllocMaxFaces = 262144;
constexpr int kNoAllocMaxVerts = 262144;
static __device__ __align__(256) float g_noalloc_scratch[2 * kNoAllocMaxFaces + kNoAllocMaxVerts];

// Device address of the scratch array, looked up per device on the first
// call that succeeds and cached from then on; a failed lookup (for example
// before the device has a usable context) is not cached, so a later call
// retries it instead of failing for the rest of the process.
static float* scratch_address(int device, tc_status* st) {
  constexpr int kMaxDevices = 64;
  static float* addr[kMaxDevices] = {};
  static std::mutex lock;
  if (device < 0 || device >= kMaxDevices) {
    *st = TC_ERR_INVALID_ARG;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(lock);
  if (!addr[device]) {
    void* p = nullptr;
    // the calling thread has `device` current here
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) == cudaSuccess) addr[device] = (float*)p;
    else (void)cudaGetLastError();  // clear the non-sticky error of the failed lookup
  }
  *st = addr[device] ? TC_OK : TC_ERR_CUDA;
  return addr[device];
}

// p = -n.sigma.n on the deformed contact face (stored winding outward) and
// its area; sigma read from the parent tet (component-major 6 x nt).
__global__ void __launch_bounds__(kBlock)
    k_face_pressure_from_sigma(const float* __restrict__ x, int nv, const float* __restrict__ sigma, int nt,
                               const int32_t* __restrict__ cfaces, const int32_t* __restrict__ cparent, int nfc,
                               float* __restrict__ face_p, float* __restrict__ face_A) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfc) return;
  const int a = cfaces[f], b = cfaces[nfc + f], c = cfaces[2 * nfc + f];
  float e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = x[d * nv + b] - x[d * nv + a];
    e2[d] = x[d * nv + c] - x[d * nv + a];
  }
  float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const float len = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const float il = len > 0.f ? 1.f / len : 0.f;
  for (int d = 0; d < 3; ++d) n[d] *= il;
  const int el = cparent[f];
  const float sxx = sigma[el], syy = sigma[(int64_t)nt + el], szz = sigma[2 * (int64_t)nt + el];
  const float sxy = sigma[3 * (int64_t)nt + el], syz = sigma[4 * (int64_t)nt + el], szx = sigma[5 * (int64_t)nt + el];
  const float t0 = sxx * n[0] + sxy * n[1] + szx * n[2];
  const float t1 = sxy * n[0] + syy * n[1] + syz * n[2];
  const float t2 = szx * n[0] + syz * n[1] + szz * n[2];
  face_p[f] = -(t0 * n[0] + t1 * n[1] + t2 * n[2]);
  face_A[f] = 0.5f * len;
}

}  // namespace tc

extern "C" tc_status tc_pressure_map_noalloc(const float* x, int32_t nv, const float* sigma, int32_t nt,
                                             const int32_t* cfaces, const int32_t* cparent,
                                             const int32_t* cface_slot, int32_t nfc, const int32_t* cv_face_off,
                                             const int32_t* cv_face_idx, int32_t nvc, const int32_t* pix_face,
                                             const float* pix_w, int32_t npix, float* out, uint8_t* mask,
                                             void* stream) {
  using namespace tc;
  if (nv < 0 || nt < 0 || nfc < 0 || nvc < 0 || npix < 0) return TC_ERR_INVALID_ARG;
  if (nfc > kNoAllocMaxFaces || nvc > kNoAllocMaxVerts) return TC_ERR_CAPACITY;
  if (npix > 0 && (!out || !pix_face || !pix_w)) return TC_ERR_INVALID_ARG;
  if (nfc > 0 && (!x || !sigma || !cfaces || !cparent || !cface_slot)) return TC_ERR_INVALID_ARG;
  if (nvc > 0 && (!cv_face_off || !cv_face_idx)) return TC_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TC_ERR_CUDA;
  tc_status st = TC_OK;
  float* scratch = scratch_address(dev, &st);
  if (st != TC_OK) return st;
  float* face_p = scratch;
  float* face_A = scratch + kNoAllocMaxFaces;
  float* vert_p = scratch + 2 * kNoAllocMaxFaces;
  cudaStream_t s = (cudaStream_t)stream;
  // every scratch entry read below is written first in the same call, so
  // nothing has to be cleared
  if (nfc > 0)
    TC_LAUNCH("k_face_pressure_from_sigma", s,
              k_face_pressure_from_sigma<<<grid_for(nfc), kBlock, 0, s>>>(x, nv, sigma, nt, cfaces, cparent, nfc,
                                                                           face_p, face_A));
  launch_vertex_avg(nvc, cv_face_off, cv_face_idx, face_p, face_A, vert_p, s);
  launch_splat(npix, pix_face, pix_w, cface_slot, nfc, vert_p, out, mask, s);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TC_ERR_CUDA;
  return TC_OK;
}
