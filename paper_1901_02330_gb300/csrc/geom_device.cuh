// Small device helpers: double3 algebra and the Dunavant degree-4 triangle
// rule (D.A. Dunavant, IJNME 21 (1985): 6 points in two (a, a, 1-2a)
// orbits; weights are fractions of the triangle's area).
#pragma once

#include <cuda_runtime.h>

namespace vem {

__device__ __forceinline__ double3 load3(const double *p, int64_t i) {
  return make_double3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}
__device__ __forceinline__ void store3(double *p, int64_t i, double3 v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}
__device__ __forceinline__ double3 add3(double3 a, double3 b) {
  return make_double3(a.x + b.x, a.y + b.y, a.z + b.z);
}
__device__ __forceinline__ double3 sub3(double3 a, double3 b) {
  return make_double3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ double3 scale3(double3 a, double s) {
  return make_double3(a.x * s, a.y * s, a.z * s);
}
__device__ __forceinline__ double dot3(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross3(double3 a, double3 b) {
  return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double norm3(double3 a) { return sqrt(dot3(a, a)); }
__device__ __forceinline__ double comp3(double3 a, int c) { return c == 0 ? a.x : (c == 1 ? a.y : a.z); }

// q-th point (barycentric l0, l1, l2) and area fraction w of the rule.
__device__ __forceinline__ void dunavant4_point(int q, double &l0, double &l1, double &l2, double &w) {
  const double a = (q < 3) ? 0.445948490915965 : 0.091576213509771;
  const double b = 1.0 - 2.0 * a;
  w = (q < 3) ? 0.223381589678011 : 0.109951743655322;
  const int r = q % 3;
  l0 = (r == 2) ? b : a;
  l1 = (r == 1) ? b : a;
  l2 = (r == 0) ? b : a;
}

// Radon's 7-point degree-5 rule: barycentric coordinates and area fraction
// of point q.
__device__ __forceinline__ void radon7_point(int q, double &l0, double &l1, double &l2, double &w) {
  const double s15 = 3.872983346207416885;   // sqrt(15)
  if (q == 0) {
    l0 = l1 = l2 = 1.0 / 3.0;
    w = 9.0 / 40.0;
    return;
  }
  const bool first = q < 4;
  const double a = first ? (6.0 - s15) / 21.0 : (6.0 + s15) / 21.0;
  w = first ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0;
  const int r = (q - 1) % 3;
  l0 = (r == 0) ? 1.0 - 2.0 * a : a;
  l1 = (r == 1) ? 1.0 - 2.0 * a : a;
  l2 = (r == 2) ? 1.0 - 2.0 * a : a;
}

// Point q of the boundary-data rule on a fan triangle: ppt = 6, Dunavant's
// degree 4 (E0 and the paper's k = 1); ppt = 7, Radon's degree 5 (k = 2,
// where g_D m^f has degree 5 for g_D in P_3).
__device__ __forceinline__ void bface_point(int ppt, int q, double &l0, double &l1, double &l2, double &w) {
  if (ppt == 7) radon7_point(q, l0, l1, l2, w);
  else dunavant4_point(q, l0, l1, l2, w);
}

}  // namespace vem
