// Clipped Voronoi (and centroidal Voronoi by Lloyd iterations) meshes of the
// unit cube, as face-based polyhedral meshes.  Input generator only: it
// computes cell shapes and seed moves, none of the discretisation.
//
// Each cell starts as the cube and is clipped by the bisector half-space of
// every seed closer than twice its current radius (the security radius:
// a farther seed cannot cut the cell).  Clipping a convex polyhedron by a
// plane: Sutherland-Hodgman on every face, and a new cap face from the
// points on the plane, ordered by angle.  The face between cells i < j is
// taken from cell i, oriented outward from i; faces whose area is below
// 1e-12 of the cell scale squared, or that only one of the two cells found,
// are dropped (they are rounding-level slivers).
//
// Build: g++ -O2 -fopenmp -shared -fPIC voronoi.cpp -o libvoronoi.so
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct Face {
  int tag;                 // neighbour seed id, or -1..-6 for the cube sides
  std::vector<V3> p;       // loop, counter-clockwise seen from outside
};

struct Cell {
  std::vector<Face> f;
};

Cell unit_cube() {
  const V3 c[8] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  Cell cell;
  auto F = [&](int tag, int a, int b, int cc, int d) { cell.f.push_back({tag, {c[a], c[b], c[cc], c[d]}}); };
  F(-1, 0, 4, 7, 3);   // x = 0, outward -x
  F(-2, 1, 2, 6, 5);   // x = 1
  F(-3, 0, 1, 5, 4);   // y = 0
  F(-4, 3, 7, 6, 2);   // y = 1
  F(-5, 0, 3, 2, 1);   // z = 0
  F(-6, 4, 5, 6, 7);   // z = 1
  return cell;
}

// Clip by {x: (x - m).nrm <= 0}; returns false if the cell vanished.
bool clip(Cell &cell, V3 m, V3 nrm, int tag, double eps) {
  bool any_out = false;
  for (auto &F : cell.f)
    for (auto &q : F.p)
      if (dot(q - m, nrm) > eps) any_out = true;
  if (!any_out) return true;
  std::vector<V3> cap;
  std::vector<Face> out;
  out.reserve(cell.f.size() + 1);
  for (auto &F : cell.f) {
    const size_t k = F.p.size();
    std::vector<double> d(k);
    for (size_t i = 0; i < k; ++i) d[i] = dot(F.p[i] - m, nrm);
    std::vector<V3> np;
    np.reserve(k + 2);
    for (size_t i = 0; i < k; ++i) {
      const size_t j = (i + 1) % k;
      const V3 a = F.p[i], b = F.p[j];
      const bool ina = d[i] <= eps, inb = d[j] <= eps;
      if (ina) {
        np.push_back(a);
        if (std::fabs(d[i]) <= eps) cap.push_back(a);
      }
      if (ina != inb && std::fabs(d[i]) > eps && std::fabs(d[j]) > eps) {
        const double t = d[i] / (d[i] - d[j]);
        const V3 q = a + t * (b - a);
        np.push_back(q);
        cap.push_back(q);
      }
    }
    if (np.size() >= 3) out.push_back({F.tag, std::move(np)});
  }
  // cap polygon: unique points on the plane, ordered counter-clockwise about nrm
  std::vector<V3> u;
  for (auto &q : cap) {
    bool dup = false;
    for (auto &w : u)
      if (norm(q - w) <= 4 * eps) {
        dup = true;
        break;
      }
    if (!dup) u.push_back(q);
  }
  if (u.size() >= 3) {
    V3 c{0, 0, 0};
    for (auto &q : u) c = c + q;
    c = (1.0 / u.size()) * c;
    V3 e1 = u[0] - c;
    e1 = (1.0 / norm(e1)) * e1;
    V3 e2 = cross(nrm, e1);
    std::vector<std::pair<double, V3>> ang;
    for (auto &q : u) ang.push_back({std::atan2(dot(q - c, e2), dot(q - c, e1)), q});
    std::sort(ang.begin(), ang.end(), [](auto &a, auto &b) { return a.first < b.first; });
    Face cf{tag, {}};
    for (auto &a : ang) cf.p.push_back(a.second);
    out.push_back(std::move(cf));
  }
  cell.f = std::move(out);
  return cell.f.size() >= 4;
}

double poly_area(const std::vector<V3> &p) {
  V3 a{0, 0, 0};
  for (size_t i = 0; i < p.size(); ++i) a = a + cross(p[i] - p[0], p[(i + 1) % p.size()] - p[0]);
  return 0.5 * norm(a);
}

// volume and barycentre of a convex cell (pyramids from an interior point)
void cell_moments(const Cell &cell, double &vol, V3 &cen) {
  V3 ref{0, 0, 0};
  int np = 0;
  for (auto &F : cell.f)
    for (auto &q : F.p) {
      ref = ref + q;
      ++np;
    }
  ref = (1.0 / np) * ref;
  vol = 0;
  cen = {0, 0, 0};
  for (auto &F : cell.f)
    for (size_t i = 1; i + 1 < F.p.size(); ++i) {
      const V3 a = F.p[0] - ref, b = F.p[i] - ref, c = F.p[i + 1] - ref;
      const double v = dot(a, cross(b, c)) / 6.0;
      vol += v;
      cen = cen + v * (0.25 * (F.p[0] + F.p[i] + F.p[i + 1] + ref));
    }
  cen = (1.0 / vol) * cen;
}

struct Grid {
  int g;
  std::vector<std::vector<int>> bins;
  explicit Grid(const std::vector<V3> &s) {
    g = std::max(1, (int)std::cbrt((double)s.size() / 2.0));
    bins.assign((size_t)g * g * g, {});
    for (int i = 0; i < (int)s.size(); ++i) bins[idx(s[i])].push_back(i);
  }
  int coord(double v) const { return std::min(g - 1, std::max(0, (int)(v * g))); }
  size_t idx(V3 p) const { return ((size_t)coord(p.x) * g + coord(p.y)) * g + coord(p.z); }
};

Cell build_cell(int i, const std::vector<V3> &s, const Grid &G, double eps) {
  Cell cell = unit_cube();
  const V3 si = s[i];
  const int cx = G.coord(si.x), cy = G.coord(si.y), cz = G.coord(si.z);
  std::vector<std::pair<double, int>> cand;
  int done_ring = -1;
  for (int ring = 0; ring <= 2 * G.g; ++ring) {
    // gather the seeds of this ring of bins
    for (int a = cx - ring; a <= cx + ring; ++a)
      for (int b = cy - ring; b <= cy + ring; ++b)
        for (int c = cz - ring; c <= cz + ring; ++c) {
          if (std::max({std::abs(a - cx), std::abs(b - cy), std::abs(c - cz)}) != ring) continue;
          if (a < 0 || b < 0 || c < 0 || a >= G.g || b >= G.g || c >= G.g) continue;
          for (int j : G.bins[((size_t)a * G.g + b) * G.g + c])
            if (j != i) cand.push_back({norm(s[j] - si), j});
        }
    // every seed within ring / g of si has been gathered
    const double reach = (double)ring / G.g;
    std::sort(cand.begin(), cand.end());
    double rmax = 0;
    for (auto &F : cell.f)
      for (auto &q : F.p) rmax = std::max(rmax, norm(q - si));
    size_t k = 0;
    for (; k < cand.size(); ++k) {
      if (cand[k].first > reach) break;
      if (cand[k].first >= 2 * rmax) break;
      const int j = cand[k].second;
      if (cand[k].first < 1e-14) continue;   // coincident seeds: no bisector
      const V3 nrm = (1.0 / cand[k].first) * (s[j] - si);
      clip(cell, 0.5 * (si + s[j]), nrm, j, eps);
      rmax = 0;
      for (auto &F : cell.f)
        for (auto &q : F.p) rmax = std::max(rmax, norm(q - si));
    }
    cand.erase(cand.begin(), cand.begin() + k);
    done_ring = ring;
    if (reach >= 2 * rmax) break;
  }
  (void)done_ring;
  return cell;
}

struct Out {
  std::vector<double> xyz;
  std::vector<int64_t> fptr{0};
  std::vector<int32_t> fv;
  std::vector<int64_t> cptr{0};
  std::vector<int32_t> cf;
  std::vector<int8_t> fbc;
  std::vector<double> seeds;
  int64_t dropped = 0;
};

}  // namespace

extern "C" {

// Build the (optionally Lloyd-relaxed) clipped Voronoi mesh of n seeds
// (coordinates in [0,1]^3, modified in place by the Lloyd steps).  Returns an
// opaque result read by voronoi_sizes / voronoi_copy, freed by voronoi_free.
void *voronoi_build(int64_t n, double *seeds, int lloyd_iters) {
  std::vector<V3> s(n);
  for (int64_t i = 0; i < n; ++i) s[i] = {seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2]};
  const double h = std::cbrt(1.0 / (double)n);
  const double eps = 1e-12 * h;
  std::vector<Cell> cells(n);
  for (int it = 0; it <= lloyd_iters; ++it) {
    Grid G(s);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) cells[i] = build_cell((int)i, s, G, eps);
    if (it == lloyd_iters) break;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double vol;
      V3 c;
      cell_moments(cells[i], vol, c);
      s[i] = c;
    }
  }
  auto *o = new Out();
  for (int64_t i = 0; i < n; ++i) {
    seeds[3 * i] = s[i].x;
    seeds[3 * i + 1] = s[i].y;
    seeds[3 * i + 2] = s[i].z;
  }
  // which (i, j) faces each side found, with their areas
  const double amin = 1e-12 * h * h;
  std::map<std::pair<int, int>, int> fid;   // (i, j) i < j -> face id
  std::vector<std::vector<std::pair<int, int>>> cellfaces(n);   // (tag, local face index)
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < (int)cells[i].f.size(); ++k) cellfaces[i].push_back({cells[i].f[k].tag, k});
  auto has_tag = [&](int64_t c, int tag) {
    for (auto &t : cellfaces[c])
      if (t.first == tag) return true;
    return false;
  };
  for (int64_t i = 0; i < n; ++i) {
    for (auto &F : cells[i].f) {
      const int j = F.tag;
      const bool bnd = j < 0;
      if (!bnd && j < i) continue;                       // taken from the lower id
      if (poly_area(F.p) < amin || (!bnd && !has_tag(j, (int)i))) {
        ++o->dropped;
        continue;
      }
      const int id = (int)o->fbc.size();
      fid[{(int)i, j}] = id;
      for (auto &q : F.p) {
        o->fv.push_back((int32_t)(o->xyz.size() / 3));
        o->xyz.push_back(q.x);
        o->xyz.push_back(q.y);
        o->xyz.push_back(q.z);
      }
      o->fptr.push_back((int64_t)o->fv.size());
      o->fbc.push_back(bnd ? 1 : 0);
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (auto &F : cells[i].f) {
      const int j = F.tag;
      std::pair<int, int> key = (j < 0 || i < j) ? std::make_pair((int)i, j) : std::make_pair(j, (int)i);
      auto it = fid.find(key);
      if (it != fid.end()) o->cf.push_back(it->second);
    }
    o->cptr.push_back((int64_t)o->cf.size());
  }
  return o;
}

void voronoi_sizes(void *r, int64_t *nv, int64_t *nf, int64_t *nfv, int64_t *nc, int64_t *ncf, int64_t *dropped) {
  auto *o = static_cast<Out *>(r);
  *nv = (int64_t)o->xyz.size() / 3;
  *nf = (int64_t)o->fbc.size();
  *nfv = (int64_t)o->fv.size();
  *nc = (int64_t)o->cptr.size() - 1;
  *ncf = (int64_t)o->cf.size();
  *dropped = o->dropped;
}

void voronoi_copy(void *r, double *xyz, int64_t *fptr, int32_t *fv, int64_t *cptr, int32_t *cf, int8_t *fbc) {
  auto *o = static_cast<Out *>(r);
  std::memcpy(xyz, o->xyz.data(), o->xyz.size() * sizeof(double));
  std::memcpy(fptr, o->fptr.data(), o->fptr.size() * sizeof(int64_t));
  std::memcpy(fv, o->fv.data(), o->fv.size() * sizeof(int32_t));
  std::memcpy(cptr, o->cptr.data(), o->cptr.size() * sizeof(int64_t));
  std::memcpy(cf, o->cf.data(), o->cf.size() * sizeof(int32_t));
  std::memcpy(fbc, o->fbc.data(), o->fbc.size() * sizeof(int8_t));
}

void voronoi_free(void *r) { delete static_cast<Out *>(r); }

}  // extern "C"
