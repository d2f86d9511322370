// Shared device helpers: lattice geometry, packed layouts, complex arithmetic.
//
// Geometry (Sec. III-A-1 site numbering, last coordinate fastest) and the
// odd-even split (Sec. III-A-2): a site with coordinates (t, z, y, x) has
// number lex = ((t*Z + z)*Y + y)*X + x and parity p = (t+z+y+x) & 1. With X
// even, the two sites lex = 2k and 2k+1 have opposite parities, so
// cb = lex >> 1 numbers the V/2 sites of each parity in increasing site order.
// Every site-indexed array on the device is in "eo order": index
// i = p * V/2 + cb (even sites first).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lqcd {

struct Geom {
  int T, Z, Y, X;
  int V, Vh;
  int XY, XYZ;
};

struct Coord {
  int t, z, y, x;
  int lex;
};

__host__ __device__ inline Geom make_geom(const int d[4]) {
  Geom g;
  g.T = d[0]; g.Z = d[1]; g.Y = d[2]; g.X = d[3];
  g.XY = g.X * g.Y;
  g.XYZ = g.XY * g.Z;
  g.V = g.XYZ * g.T;
  g.Vh = g.V / 2;
  return g;
}

// (parity, cb) -> coordinates.
__device__ __forceinline__ Coord site_coords(const Geom& g, int p, int cb) {
  Coord c;
  int l2 = cb << 1;
  int x0 = l2 % g.X;
  int r = l2 / g.X;
  c.y = r % g.Y;
  r /= g.Y;
  c.z = r % g.Z;
  c.t = r / g.Z;
  c.x = x0 + ((p + c.t + c.z + c.y) & 1);
  c.lex = l2 - x0 + c.x;
  return c;
}

// Site number of the neighbour x + mu-hat (dir = +1) or x - mu-hat (dir = -1), periodic wrap.
template <int MU, int DIR>
__device__ __forceinline__ int neighbour_lex(const Geom& g, const Coord& c) {
  if (MU == 0) {
    if (DIR > 0) return (c.t == g.T - 1) ? c.lex - (g.T - 1) * g.XYZ : c.lex + g.XYZ;
    return (c.t == 0) ? c.lex + (g.T - 1) * g.XYZ : c.lex - g.XYZ;
  } else if (MU == 1) {
    if (DIR > 0) return (c.z == g.Z - 1) ? c.lex - (g.Z - 1) * g.XY : c.lex + g.XY;
    return (c.z == 0) ? c.lex + (g.Z - 1) * g.XY : c.lex - g.XY;
  } else if (MU == 2) {
    if (DIR > 0) return (c.y == g.Y - 1) ? c.lex - (g.Y - 1) * g.X : c.lex + g.X;
    return (c.y == 0) ? c.lex + (g.Y - 1) * g.X : c.lex - g.X;
  } else {
    if (DIR > 0) return (c.x == g.X - 1) ? c.lex - (g.X - 1) : c.lex + 1;
    return (c.x == 0) ? c.lex + (g.X - 1) : c.lex - 1;
  }
}

// Packed spinor layout: complex index of (site i, component c in 0..11, rhs r)
// for a block with nrhs rhs and a site tile of 2^log_s sites:
//   ((i >> log_s) * 12 + c) * (S * nrhs) + (i & (S-1)) * nrhs + r.
// The rhs index is innermost (Eq. (2)'s rows stored rhs-fastest), so the b
// threads of one site read one contiguous run per component.
struct PackedLayout {
  int nrhs;
  int log_s;
  __host__ __device__ __forceinline__ int64_t index(int64_t i, int c, int r) const {
    const int64_t S = int64_t(1) << log_s;
    return ((i >> log_s) * 12 + c) * (S * nrhs) + (i & (S - 1)) * nrhs + r;
  }
};

// ------------------------------------------------------------------ complex helpers

template <typename Real> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im) {
  C z; z.x = re; z.y = im; return z;
}

__host__ __device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d2(double2 a) { return a; }

// Error-status flags written by device code (bitmask in a device int).
enum : int { DEV_ERR_SINGULAR = 1, DEV_ERR_NONFINITE = 2 };

}  // namespace lqcd
