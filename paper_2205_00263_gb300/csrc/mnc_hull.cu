// Host generator of multi-neuron constraints over groups of k = 3 neurons.
//
// The paper takes its constraints from PRIMA (Sec. 2.3; Sec. 3.1, enforcing
// multi-neuron constraints) and gives no generator: any linear constraint that
// holds on the joint (z, zhat) space of a ReLU layer is admissible.  This
// library's construction, for one group G = (j0, j1, j2) of unstable neurons:
//
//  1. the octahedron O = {x : d . x >= lb_d} over-approximates zhat_G, with
//     lb_d the DeepPoly lower bound of d . zhat_G for the 26 directions
//     d in {-1, 0, 1}^3 \ {0} (computed on the device at the root);
//  2. in each of the 8 orthants the ReLU is linear, so the graph of relu over
//     O is the union of the lifted orthant pieces {(relu(x), x) : x in O and
//     orthant}; their convex hull is spanned by the lifted vertices of the
//     3-D polytopes O and orthant;
//  3. the facets n_y . y + n_x . x <= p of that 6-D hull are the extreme rays
//     of the cone {(a, b) : a . v <= b for every lifted vertex v}, found by the
//     double-description method (rays updated one constraint at a time, new
//     rays only from adjacent pairs, adjacency by the common tight set);
//  4. each facet normal is scaled to unit length, its offset re-tightened to
//     the exact support max_v a . v, and facets that involve a single neuron
//     are dropped (the single-neuron relaxation already holds them).
//
// Everything here is FP64 host arithmetic; nothing runs on the device.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mnbab.h"
#include "mnbab_internal.h"

namespace mnbab {

namespace {

using Vec3 = std::array<double, 3>;
using Pt6 = std::array<double, 6>;
constexpr int HD = 7;  // homogeneous facet coordinates (a in R^6, b)

Vec3 cross(const Vec3& a, const Vec3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double dot3(const Vec3& a, const Vec3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Vertices of {x : n_i . x >= b_i for all i} in 3-D: intersections of plane
// triples that satisfy every inequality.
void polytope_vertices(const std::vector<Vec3>& n, const std::vector<double>& b,
                       std::vector<Vec3>& out) {
  const int m = (int)n.size();
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const Vec3 cij = cross(n[i], n[j]);
      for (int k = j + 1; k < m; ++k) {
        const double det = dot3(n[k], cij);
        if (std::fabs(det) < 1e-12) continue;
        // Cramer's rule with cross products: x = (b_i (n_j x n_k) + b_j (n_k x n_i) + b_k (n_i x n_j)) / det
        const Vec3 cjk = cross(n[j], n[k]), cki = cross(n[k], n[i]);
        Vec3 x;
        for (int c = 0; c < 3; ++c) x[c] = (b[i] * cjk[c] + b[j] * cki[c] + b[k] * cij[c]) / det;
        bool ok = true;
        for (int q = 0; q < m && ok; ++q)
          ok = dot3(n[q], x) - b[q] >= -1e-9 * (1.0 + std::fabs(b[q]));
        if (!ok) continue;
        bool dup = false;
        for (const Vec3& y : out)
          if (std::fabs(y[0] - x[0]) + std::fabs(y[1] - x[1]) + std::fabs(y[2] - x[2]) <
              1e-10 * (1.0 + std::fabs(x[0]) + std::fabs(x[1]) + std::fabs(x[2]))) {
            dup = true;
            break;
          }
        if (!dup) out.push_back(x);
      }
    }
}

// ---- double description -------------------------------------------------
struct Ray {
  double v[HD];
  std::vector<uint64_t> tight;  // constraints with A_i . v = 0
};

bool has(const std::vector<uint64_t>& s, int i) { return (s[i >> 6] >> (i & 63)) & 1u; }
void put(std::vector<uint64_t>& s, int i) { s[i >> 6] |= uint64_t(1) << (i & 63); }
int count(const std::vector<uint64_t>& s) {
  int c = 0;
  for (uint64_t w : s) c += __builtin_popcountll(w);
  return c;
}
bool subset(const std::vector<uint64_t>& a, const std::vector<uint64_t>& b) {  // a within b
  for (size_t w = 0; w < a.size(); ++w)
    if (a[w] & ~b[w]) return false;
  return true;
}

void normalize(double* v) {
  double s = 0.0;
  for (int c = 0; c < HD; ++c) s += v[c] * v[c];
  s = std::sqrt(s);
  if (s > 0)
    for (int c = 0; c < HD; ++c) v[c] /= s;
}

// Facets (a, b), a . x <= b, of the convex hull of pts (full-dimensional in
// R^6): the extreme rays of the cone {y : A y >= 0}, A_i = (-v_i, 1).  Returns
// false when the points span less than 6 dimensions.
bool hull_facets(const std::vector<Pt6>& pts, std::vector<std::array<double, HD>>& facets) {
  const int m = (int)pts.size();
  if (m < HD) return false;
  std::vector<std::array<double, HD>> A(m);
  double scale = 1.0;
  for (int i = 0; i < m; ++i) {
    for (int c = 0; c < 6; ++c) {
      A[i][c] = -pts[i][c];
      scale = std::max(scale, std::fabs(pts[i][c]));
    }
    A[i][6] = 1.0;
  }
  // a first basis of HD independent constraints (Gram-Schmidt on the rows)
  std::vector<int> basis;
  std::vector<std::array<double, HD>> q;
  for (int i = 0; i < m && (int)basis.size() < HD; ++i) {
    std::array<double, HD> r = A[i];
    double n0 = 0.0;
    for (int c = 0; c < HD; ++c) n0 += r[c] * r[c];
    for (const auto& e : q) {
      double d = 0.0;
      for (int c = 0; c < HD; ++c) d += r[c] * e[c];
      for (int c = 0; c < HD; ++c) r[c] -= d * e[c];
    }
    double n1 = 0.0;
    for (int c = 0; c < HD; ++c) n1 += r[c] * r[c];
    if (n1 <= 1e-18 * n0) continue;
    const double inv = 1.0 / std::sqrt(n1);
    for (int c = 0; c < HD; ++c) r[c] *= inv;
    q.push_back(r);
    basis.push_back(i);
  }
  if ((int)basis.size() < HD) return false;
  // initial rays: the columns of the basis matrix's inverse (Gauss-Jordan)
  double M[HD][2 * HD];
  for (int r = 0; r < HD; ++r)
    for (int c = 0; c < HD; ++c) {
      M[r][c] = A[basis[r]][c];
      M[r][HD + c] = r == c ? 1.0 : 0.0;
    }
  for (int col = 0; col < HD; ++col) {
    int piv = col;
    for (int r = col + 1; r < HD; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (std::fabs(M[piv][col]) < 1e-14) return false;
    if (piv != col)
      for (int c = 0; c < 2 * HD; ++c) std::swap(M[piv][c], M[col][c]);
    const double d = M[col][col];
    for (int c = 0; c < 2 * HD; ++c) M[col][c] /= d;
    for (int r = 0; r < HD; ++r) {
      if (r == col || M[r][col] == 0.0) continue;
      const double f = M[r][col];
      for (int c = 0; c < 2 * HD; ++c) M[r][c] -= f * M[col][c];
    }
  }
  const int words = (m + 63) / 64;
  std::vector<Ray> rays(HD);
  for (int j = 0; j < HD; ++j) {
    for (int c = 0; c < HD; ++c) rays[j].v[c] = M[c][HD + j];
    normalize(rays[j].v);
    rays[j].tight.assign(words, 0);
    for (int k = 0; k < HD; ++k)
      if (k != j) put(rays[j].tight, basis[k]);
  }
  std::vector<char> in_basis(m, 0);
  for (int i : basis) in_basis[i] = 1;
  const double tol = 1e-10 * (1.0 + scale);
  std::vector<double> s;
  std::vector<int> pos, neg;
  std::vector<Ray> next;
  for (int i = 0; i < m; ++i) {
    if (in_basis[i]) continue;
    const int nr = (int)rays.size();
    s.assign(nr, 0.0);
    pos.clear();
    neg.clear();
    for (int r = 0; r < nr; ++r) {
      double v = 0.0;
      for (int c = 0; c < HD; ++c) v += A[i][c] * rays[r].v[c];
      s[r] = v;
      if (v > tol) pos.push_back(r);
      else if (v < -tol) neg.push_back(r);
    }
    if (neg.empty()) {
      for (int r = 0; r < nr; ++r)
        if (std::fabs(s[r]) <= tol) put(rays[r].tight, i);
      continue;
    }
    next.clear();
    for (int r = 0; r < nr; ++r) {
      if (s[r] < -tol) continue;
      next.push_back(rays[r]);
      if (s[r] <= tol) put(next.back().tight, i);
    }
    std::vector<uint64_t> common(words);
    for (int p : pos)
      for (int g : neg) {
        for (int w = 0; w < words; ++w) common[w] = rays[p].tight[w] & rays[g].tight[w];
        if (count(common) < HD - 2) continue;
        // adjacent iff no third ray is tight on every common constraint
        bool adj = true;
        for (int r = 0; r < nr && adj; ++r)
          if (r != p && r != g && subset(common, rays[r].tight)) adj = false;
        if (!adj) continue;
        Ray w;
        for (int c = 0; c < HD; ++c) w.v[c] = s[p] * rays[g].v[c] - s[g] * rays[p].v[c];
        normalize(w.v);
        w.tight = common;
        put(w.tight, i);
        next.push_back(std::move(w));
      }
    rays.swap(next);
  }
  facets.clear();
  for (const Ray& r : rays) {
    std::array<double, HD> f;
    for (int c = 0; c < HD; ++c) f[c] = r.v[c];
    facets.push_back(f);
  }
  return true;
}

}  // namespace

// Constraint rows of one group from its 26 octahedral lower bounds (see the
// file comment).  Returns false when the group gives no rows (degenerate).
bool mnc_group_rows(const double* oct_lb, std::vector<MncRow>& rows) {
  rows.clear();
  std::vector<Vec3> dirs;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int c = -1; c <= 1; ++c)
        if (a || b || c) dirs.push_back({(double)a, (double)b, (double)c});
  std::vector<Pt6> pts;
  for (int o = 0; o < 8; ++o) {
    const double sg[3] = {(o & 4) ? 1.0 : -1.0, (o & 2) ? 1.0 : -1.0, (o & 1) ? 1.0 : -1.0};
    std::vector<Vec3> n(dirs);
    std::vector<double> b(oct_lb, oct_lb + 26);
    for (int k = 0; k < 3; ++k) {
      Vec3 e = {0.0, 0.0, 0.0};
      e[k] = sg[k];
      n.push_back(e);
      b.push_back(0.0);
    }
    std::vector<Vec3> vs;
    polytope_vertices(n, b, vs);
    for (const Vec3& x : vs) {
      Pt6 p;
      for (int k = 0; k < 3; ++k) {
        p[k] = sg[k] > 0 ? std::max(x[k], 0.0) : 0.0;  // relu is linear in the orthant
        p[3 + k] = x[k];
      }
      bool dup = false;
      for (const Pt6& q : pts) {
        double dd = 0.0, mag = 1.0;
        for (int c = 0; c < 6; ++c) {
          dd += std::fabs(p[c] - q[c]);
          mag += std::fabs(p[c]);
        }
        if (dd < 1e-10 * mag) {
          dup = true;
          break;
        }
      }
      if (!dup) pts.push_back(p);
    }
  }
  std::vector<std::array<double, HD>> facets;
  if (!hull_facets(pts, facets)) return false;
  for (const auto& f : facets) {
    double na = 0.0;
    for (int c = 0; c < 6; ++c) na += f[c] * f[c];
    na = std::sqrt(na);
    if (na < 1e-12) continue;
    MncRow r;
    int support = 0;
    for (int k = 0; k < 3; ++k) {
      r.P[k] = f[k] / na;
      r.Ph[k] = f[3 + k] / na;
      if (std::fabs(r.P[k]) > 1e-9 || std::fabs(r.Ph[k]) > 1e-9) ++support;
    }
    if (support <= 1) continue;
    double sup = -INFINITY;
    for (const Pt6& p : pts) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += r.P[k] * p[k] + r.Ph[k] * p[3 + k];
      sup = std::max(sup, v);
    }
    r.p = sup;
    rows.push_back(r);
  }
  return !rows.empty();
}

}  // namespace mnbab

extern "C" mnbab_status mnbab_mnc_group(const double* oct_lb, int32_t max_rows, double* P,
                                        double* Phat, double* p, int32_t* n_out) {
  if (!oct_lb || !n_out || max_rows < 0 || (max_rows > 0 && (!P || !Phat || !p)))
    return MNBAB_E_INVALID_ARG;
  for (int i = 0; i < 26; ++i)
    if (!std::isfinite(oct_lb[i])) return MNBAB_E_INVALID_ARG;
  std::vector<mnbab::MncRow> rows;
  mnbab::mnc_group_rows(oct_lb, rows);
  *n_out = (int32_t)rows.size();
  if ((int)rows.size() > max_rows) return MNBAB_E_BUDGET;
  for (size_t r = 0; r < rows.size(); ++r) {
    for (int k = 0; k < 3; ++k) {
      P[3 * r + k] = rows[r].P[k];
      Phat[3 * r + k] = rows[r].Ph[k];
    }
    p[r] = rows[r].p;
  }
  return MNBAB_OK;
}
