// Pocket map re-layout on the device: for every cell of every atom-type map,
// the 8 corner node values stored contiguously (x fastest, then y, then z),
// in FP32 or rounded to BF16 / FP16 (round to nearest even).  One
// interpolation then reads a single 32 B (FP32) or 16 B (16-bit) vector
// instead of eight scattered scalars.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ligate_internal.h"

namespace ligate {

template <int KIND>  // 0 = FP32, 1 = BF16, 2 = FP16
__global__ void corner_pack_kernel(const float *__restrict__ plain, int n_types, int nx, int ny,
                                   int nz, void *__restrict__ out) {
  const long long cells = (long long)(nx - 1) * (ny - 1) * (nz - 1);
  const long long total = cells * n_types;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const long long t = c / cells, r = c - t * cells;
    const int ix = (int)(r % (nx - 1));
    const int iy = (int)((r / (nx - 1)) % (ny - 1));
    const int iz = (int)(r / ((long long)(nx - 1) * (ny - 1)));
    const float *m = plain + t * (long long)nx * ny * nz + ((long long)iz * ny + iy) * nx + ix;
    const long long sy = nx, sz = (long long)nx * ny;
    float v[8] = {m[0], m[1], m[sy], m[sy + 1], m[sz], m[sz + 1], m[sz + sy], m[sz + sy + 1]};
    if (KIND == 0) {
      float4 *o = reinterpret_cast<float4 *>(out) + 2 * c;
      o[0] = make_float4(v[0], v[1], v[2], v[3]);
      o[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
      uint32_t wv[4];
      for (int q = 0; q < 4; ++q) {
        uint16_t lo, hi;
        if (KIND == 1) {
          lo = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * q]));
          hi = __bfloat16_as_ushort(__float2bfloat16_rn(v[2 * q + 1]));
        } else {
          lo = __half_as_ushort(__float2half_rn(v[2 * q]));
          hi = __half_as_ushort(__float2half_rn(v[2 * q + 1]));
        }
        wv[q] = (uint32_t)lo | ((uint32_t)hi << 16);
      }
      reinterpret_cast<uint4 *>(out)[c] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
  }
}

cudaError_t launch_corner_pack(const float *plain, int n_types, int nx, int ny, int nz,
                               int out_kind, void *out, cudaStream_t s) {
  const int block = 256, grid = 152 * 8;
  switch (out_kind) {
    case 0: corner_pack_kernel<0><<<grid, block, 0, s>>>(plain, n_types, nx, ny, nz, out); break;
    case 1: corner_pack_kernel<1><<<grid, block, 0, s>>>(plain, n_types, nx, ny, nz, out); break;
    default: corner_pack_kernel<2><<<grid, block, 0, s>>>(plain, n_types, nx, ny, nz, out); break;
  }
  return cudaGetLastError();
}

}  // namespace ligate
