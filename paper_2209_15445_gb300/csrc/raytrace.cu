// Ray tracing of the geometry (paper Sec. 2.1: navigation was validated on ray-traced
// images, GPU against CPU and single against double precision). One thread per pixel of an
// orthographic camera: the ray enters the world analytically and then crosses volume after
// volume with the transport's own locate and straight_distance, in FP64 or with FP32
// distances (FP64 positions, as in the split form). Per pixel: the mass thickness traversed
// (g/cm^2) and the number of volumes entered. The image lives in device memory.
#include <cuda_runtime.h>

#include "device.cuh"
#include "layout.h"

namespace adept {

// entry of the ray p + t u (t >= 0) into the world, snapped onto the entry face
__device__ bool world_entry(const GeoView& g, const double p[3], const double u[3], double q[3]) {
  double t0 = 0.0, t1 = 1e300;
  int face = -1;  // 0/1/2: axis of the entry plane (box) or z cap; 3: the cylinder
  double fval = 0.0;
  if (g.kind == 0) {
    const double lo[3] = {-g.half_xy, -g.half_xy, g.bnd[0]};
    const double hi[3] = {g.half_xy, g.half_xy, g.bnd[g.n_vol]};
    for (int a = 0; a < 3; ++a) {
      if (u[a] == 0.0) {
        if (p[a] < lo[a] || p[a] > hi[a]) return false;
        continue;
      }
      double ta = (lo[a] - p[a]) / u[a], tb = (hi[a] - p[a]) / u[a];
      double va = lo[a], vb = hi[a];
      if (ta > tb) { double x = ta; ta = tb; tb = x; x = va; va = vb; vb = x; }
      if (ta > t0) { t0 = ta; face = a; fval = va; }
      if (tb < t1) t1 = tb;
    }
  } else {
    const double R = g.bnd[g.n_vol - 1];
    const double a = u[0] * u[0] + u[1] * u[1], b = p[0] * u[0] + p[1] * u[1];
    const double cc = p[0] * p[0] + p[1] * p[1] - R * R;
    if (a > 0.0) {
      const double D = b * b - a * cc;
      if (D < 0.0) return false;
      const double sq = sqrt(D);
      const double ta = (-b - sq) / a, tb = (-b + sq) / a;
      if (ta > t0) { t0 = ta; face = 3; }
      if (tb < t1) t1 = tb;
    } else if (cc > 0.0) {
      return false;
    }
    if (u[2] != 0.0) {
      double ta = (-g.half_z - p[2]) / u[2], tb = (g.half_z - p[2]) / u[2];
      double va = -g.half_z, vb = g.half_z;
      if (ta > tb) { double x = ta; ta = tb; tb = x; x = va; va = vb; vb = x; }
      if (ta > t0) { t0 = ta; face = 2; fval = va; }
      if (tb < t1) t1 = tb;
    } else if (fabs(p[2]) > g.half_z) {
      return false;
    }
  }
  if (!(t0 <= t1)) return false;
  for (int a = 0; a < 3; ++a) q[a] = p[a] + t0 * u[a];
  if (face >= 0 && face < 3) q[face] = fval;
  if (face == 3) {
    const double R = g.bnd[g.n_vol - 1], r = sqrt(q[0] * q[0] + q[1] * q[1]);
    if (r > 0.0) { q[0] *= R / r; q[1] *= R / r; }
  }
  return true;
}

template <class R>
__global__ void k_raytrace(Params P, RayCam cam, int nx, int ny, int row0, int rows, double* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)nx * rows) return;
  const int i = (int)(k % nx), j = row0 + (int)(k / nx);
  const double a = ((i + 0.5) / nx - 0.5) * cam.width, b = ((j + 0.5) / ny - 0.5) * cam.height;
  const double p[3] = {cam.o[0] + a * cam.right[0] + b * cam.up[0], cam.o[1] + a * cam.right[1] + b * cam.up[1],
                       cam.o[2] + a * cam.right[2] + b * cam.up[2]};
  double q[3], mass = 0.0, n = 0.0;
  if (world_entry(P.geo, p, cam.d, q)) {
    const R u[3] = {(R)cam.d[0], (R)cam.d[1], (R)cam.d[2]};
    int vol = locate(P.geo, q[0], q[1], q[2], cam.d[0], cam.d[1], cam.d[2]);
    for (int c = 0; vol >= 0 && c < 100000; ++c) {
      n += 1.0;
      int next;
      const R s = straight_distance<R>(P.geo, q[0], q[1], q[2], u, vol, &next);
      const int m = __ldg(P.geo.vol_mat + vol);
      if (m >= 0) mass += P.mat[m].rho * to_d<R>(s) * 0.1;
      q[0] += to_d<R>(s * u[0]);
      q[1] += to_d<R>(s * u[1]);
      q[2] += to_d<R>(s * u[2]);
      if (P.geo.kind == 0 && next >= 0) q[2] = __ldg(P.geo.bnd + (cam.d[2] > 0.0 ? vol + 1 : vol));
      vol = next;
    }
  }
  out[2 * k] = mass;
  out[2 * k + 1] = n;
}

cudaError_t launch_raytrace(const Params& P, int prec, const RayCam& cam, int nx, int ny, int row0, int rows,
                            double* out, cudaStream_t st) {
  const long long n = (long long)nx * rows;
  if (n <= 0) return cudaSuccess;
  const int B = 128;
  const unsigned grid = (unsigned)((n + B - 1) / B);
  if (prec) k_raytrace<float><<<grid, B, 0, st>>>(P, cam, nx, ny, row0, rows, out);
  else k_raytrace<double><<<grid, B, 0, st>>>(P, cam, nx, ny, row0, rows, out);
  return cudaGetLastError();
}

}  // namespace adept
