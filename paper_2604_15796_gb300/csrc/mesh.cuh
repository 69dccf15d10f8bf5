// Inversion mesh <-> forward mesh (Sec. IV: the contrast is inverted on a
// mesh coarser than the forward mesh).  An inversion cell covers r x r (x r)
// forward pixels (ry = 1 along y in 2D) with a constant contrast:
// prolongation copies the cell's value, restriction (its adjoint) sums the
// cell's pixels in a fixed order.
#pragma once

#include "common.cuh"

namespace fwi {

// dst[n] (forward mesh, field precision) = src[cell(n)] (inversion mesh)
template <typename T>
__global__ void prolong_kernel(cplx<T>* __restrict__ dst, const double2* __restrict__ src,
                               int nx, int ny, int r, int ry, long long N) {
  const int inx = nx / r, iny = ny / ry;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx);
    const long long q = i / nx;
    const int iy = (int)(q % ny);
    const int iz = (int)(q / ny);
    const double2 v = src[((long long)(iz / r) * iny + iy / ry) * inx + ix / r];
    dst[i] = mk<T>((T)v.x, (T)v.y);
  }
}

// dst[j] (inversion mesh) = sum of src over the forward pixels of cell j
static __global__ void restrict_kernel(double2* __restrict__ dst, const double2* __restrict__ src,
                                       int nx, int ny, int r, int ry, long long Ninv) {
  const int inx = nx / r, iny = ny / ry;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < Ninv;
       j += (long long)gridDim.x * blockDim.x) {
    const int jx = (int)(j % inx);
    const long long q = j / inx;
    const int jy = (int)(q % iny);
    const int jz = (int)(q / iny);
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < r; ++c)
      for (int b = 0; b < ry; ++b)
        for (int a = 0; a < r; ++a) {
          const double2 v =
              src[((long long)(jz * r + c) * ny + (jy * ry + b)) * nx + (jx * r + a)];
          sx += v.x;
          sy += v.y;
        }
    dst[j] = make_double2(sx, sy);
  }
}

}  // namespace fwi
