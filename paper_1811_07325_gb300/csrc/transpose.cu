// transpose.cu -- in-place transpose of square leaf planes, for the optional
// K-major layout of the 3xTF32 B operand: the TF32 B planes written
// row-major (K x N) by the divide kernel are turned into N x K here.  Each block swaps
// a 32 x 32 tile with its mirror tile through shared memory (diagonal tiles
// transpose in place); reads and writes are coalesced along rows.
#include "stark_internal.h"

namespace stark {
namespace {

constexpr int TT = 32;

__global__ void __launch_bounds__(256) transpose_planes_kernel(float* planes, int64_t L) {
  __shared__ float a[TT][TT + 1];
  __shared__ float b[TT][TT + 1];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;  // each unordered tile pair once
  float* P = planes + (int64_t)blockIdx.z * L * L;
  const int tx = threadIdx.x % TT, ty = threadIdx.x / TT;  // 32 x 8
  const int64_t r0 = (int64_t)ti * TT, c0 = (int64_t)tj * TT;
#pragma unroll
  for (int k = 0; k < TT; k += 8) {
    a[ty + k][tx] = P[(r0 + ty + k) * L + c0 + tx];
    if (ti != tj) b[ty + k][tx] = P[(c0 + ty + k) * L + r0 + tx];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TT; k += 8) {
    // tile (tj, ti) <- a^T ; tile (ti, tj) <- b^T
    P[(c0 + ty + k) * L + r0 + tx] = a[tx][ty + k];
    if (ti != tj) P[(r0 + ty + k) * L + c0 + tx] = b[tx][ty + k];
  }
}

}  // namespace

cudaError_t launch_transpose_planes(float* planes, int64_t L, int64_t count, cudaStream_t s) {
  if (L % TT != 0 || count <= 0) return count == 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (L / TT > 65535 || count > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(L / TT), (unsigned)(L / TT), (unsigned)count);
  transpose_planes_kernel<<<grid, 256, 0, s>>>(planes, L);
  count_launch();
  return cudaGetLastError();
}

}  // namespace stark
