// Host-side mesh pipeline: validation, periodic identification, interface-node
// doubling, interface faces, the shared CSR pattern and the slot-sorted
// element-contribution lists used by the deterministic assembly kernels.
//
// Paper: PUFEM with one nodal copy per compartment (Appendix A, Eq. phase_func
// and the broken inner product (.,.)_{Omega_0 u Omega_1}); interface jump term
// kappa <[U],[v]> (Appendix B, Eq. loadvec); master-slave periodicity
// (Section 2, Eq. btpde_bc).
#include <algorithm>
#include <atomic>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <thread>

#include "bt_internal.h"

namespace bt {
namespace {

template <class F>
void parallel_for(int64_t n, F&& fn) {
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, n / 4096));
  if (nt <= 1) {
    fn(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([&fn, b, e] { fn(b, e); });
  }
  for (auto& x : th) x.join();
}

double signed_volume(const double* a, const double* b, const double* c, const double* d) {
  double e1[3], e2[3], e3[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = b[k] - a[k];
    e2[k] = c[k] - a[k];
    e3[k] = d[k] - a[k];
  }
  double cx = e1[1] * e2[2] - e1[2] * e2[1];
  double cy = e1[2] * e2[0] - e1[0] * e2[2];
  double cz = e1[0] * e2[1] - e1[1] * e2[0];
  return (cx * e3[0] + cy * e3[1] + cz * e3[2]) / 6.0;
}

int validate(const HostMesh& m, std::string& msg) {
  if (m.n_nodes <= 0 || m.n_tets <= 0 || m.n_cmpt <= 0) {
    msg = "empty mesh";
    return BT_EINVAL;
  }
  if (m.nv < 2 || m.nv > 4) {
    msg = "elements must be segments, triangles or tetrahedra";
    return BT_EINVAL;
  }
  if (m.nv == 3 && (m.pmask & 4u)) {
    msg = "a 2-D mesh has no periodic z axis";
    return BT_EINVAL;
  }
  if (m.nv == 2 && m.pmask) {
    msg = "a 1-D manifold mesh has no periodic axes";
    return BT_EINVAL;
  }
  if (m.surface && (m.nv != 3 || m.pmask)) {
    msg = "a surface mesh has triangles and no periodic axes";
    return BT_EINVAL;
  }
  if (m.n_nodes >= (int64_t(1) << 31) || m.n_tets >= (int64_t(1) << 27)) {
    msg = "mesh too large for 32-bit element indexing";
    return BT_EINVAL;
  }
  for (int k = 0; k < 3; ++k)
    if (!(m.hi[k] > m.lo[k]) || !std::isfinite(m.lo[k]) || !std::isfinite(m.hi[k])) {
      msg = "box_hi must exceed box_lo";
      return BT_EINVAL;
    }
  for (int32_t c = 0; c < m.n_cmpt; ++c) {
    if (!(m.D[c] >= 0.0) || !std::isfinite(m.D[c])) {
      msg = "D_cmpt must be finite and >= 0";
      return BT_EINVAL;
    }
    if (!(m.kappa[c] >= 0.0)) {  // +inf allowed, NaN rejected
      msg = "kappa_cmpt must be >= 0 (inf = no membrane)";
      return BT_EINVAL;
    }
  }
  for (int64_t i = 0; i < 3 * m.n_nodes; ++i)
    if (!std::isfinite(m.xyz[i])) {
      msg = "non-finite node coordinate";
      return BT_EINVAL;
    }
  const char* what = m.nv == 4 ? "tetrahedron " : m.nv == 3 ? "triangle " : "segment ";
  if (m.surface) what = "surface triangle ";
  for (int64_t t = 0; t < m.n_tets; ++t) {
    const int32_t* v = &m.tets[m.nv * t];
    for (int a = 0; a < m.nv; ++a)
      if (v[a] < 0 || v[a] >= m.n_nodes) {
        msg = what + std::to_string(t) + " has a node id out of range";
        return BT_EINVAL;
      }
    if (m.tet_cmpt[t] < 0 || m.tet_cmpt[t] >= m.n_cmpt) {
      msg = what + std::to_string(t) + " has a compartment id out of range";
      return BT_EINVAL;
    }
    double vol;
    if (m.nv == 4) {
      vol = signed_volume(&m.xyz[3 * v[0]], &m.xyz[3 * v[1]], &m.xyz[3 * v[2]], &m.xyz[3 * v[3]]);
    } else if (m.surface) {  // area of a triangle in 3-D (no orientation)
      const double* a = &m.xyz[3 * v[0]];
      const double* b = &m.xyz[3 * v[1]];
      const double* c = &m.xyz[3 * v[2]];
      const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      const double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2], n2 = u[0] * w[1] - u[1] * w[0];
      vol = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    } else if (m.nv == 2) {  // length of a segment (no orientation)
      const double* a = &m.xyz[3 * v[0]];
      const double* b = &m.xyz[3 * v[1]];
      vol = std::sqrt((b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) + (b[2] - a[2]) * (b[2] - a[2]));
    } else {  // signed area in the xy plane (counter-clockwise positive)
      const double* a = &m.xyz[3 * v[0]];
      const double* b = &m.xyz[3 * v[1]];
      const double* c = &m.xyz[3 * v[2]];
      vol = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));
    }
    if (!(vol > 0.0)) {
      msg = what + std::to_string(t) + " is degenerate or inverted (signed measure " + std::to_string(vol) + ")";
      return BT_EINVAL;
    }
  }
  return BT_OK;
}

// Master node of every node: on a periodic axis, a node on the high face is
// the node on the low face with equal other coordinates; the master of a
// group of identified nodes is its smallest index.
int periodic_identify(HostMesh& m, std::string& msg) {
  const int64_t n = m.n_nodes;
  m.master.resize(n);
  std::iota(m.master.begin(), m.master.end(), 0);
  if (m.pmask == 0) return BT_OK;
  double ext = 0;
  for (int k = 0; k < 3; ++k) ext = std::max(ext, m.hi[k] - m.lo[k]);
  const double tol = 1e-9 * ext;
  std::vector<std::array<int64_t, 3>> key(n);
  int64_t n_hi = 0, n_lo = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      double x = m.xyz[3 * i + k];
      if ((m.pmask >> k) & 1u) {
        if (std::fabs(x - m.hi[k]) < tol) {
          x = m.lo[k];
          ++n_hi;
        } else if (std::fabs(x - m.lo[k]) < tol) {
          ++n_lo;
        }
      }
      key[i][k] = (int64_t)std::llround(x / tol);
    }
  if (n_hi != n_lo) {
    msg = "periodic faces do not match (different node counts on the low and high faces)";
    return BT_EINVAL;
  }
  std::vector<int32_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
    return key[a] != key[b] ? key[a] < key[b] : a < b;
  });
  int64_t i = 0;
  while (i < n) {
    int64_t j = i + 1;
    while (j < n && key[ord[j]] == key[ord[i]]) ++j;
    for (int64_t k = i; k < j; ++k) m.master[ord[k]] = ord[i];  // ord[i] is the smallest index
    i = j;
  }
  return BT_OK;
}

// One dof per (master node, compartment) pair present in some tetrahedron of
// that compartment, numbered in increasing (node, compartment) order.
void double_interface_nodes(HostMesh& m) {
  const int64_t n = m.n_nodes;
  std::vector<int32_t> first(n, -1);
  std::vector<std::pair<int32_t, int32_t>> extra;
  const int nv = m.nv;
  for (int64_t t = 0; t < m.n_tets; ++t) {
    int32_t c = m.tet_cmpt[t];
    for (int a = 0; a < nv; ++a) {
      int32_t v = m.master[m.tets[nv * t + a]];
      if (first[v] < 0)
        first[v] = c;
      else if (first[v] != c)
        extra.emplace_back(v, c);
    }
  }
  std::sort(extra.begin(), extra.end());
  extra.erase(std::unique(extra.begin(), extra.end()), extra.end());
  // per node: sorted list of its compartments
  std::vector<int64_t> base(n + 1, 0);
  std::vector<int32_t> cnt(n, 0);
  for (int64_t v = 0; v < n; ++v) cnt[v] = first[v] >= 0 ? 1 : 0;
  for (auto& e : extra) cnt[e.first]++;
  for (int64_t v = 0; v < n; ++v) base[v + 1] = base[v] + cnt[v];
  m.n_dof = base[n];
  m.dof_node.resize(m.n_dof);
  m.dof_cmpt.resize(m.n_dof);
  size_t ei = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (cnt[v] == 0) continue;
    int32_t* cl = &m.dof_cmpt[base[v]];
    int k = 0;
    cl[k++] = first[v];
    while (ei < extra.size() && extra[ei].first == v) cl[k++] = extra[ei++].second;
    std::sort(cl, cl + k);
    for (int j = 0; j < k; ++j) m.dof_node[base[v] + j] = (int32_t)v;
  }
  m.tet_dof.resize(nv * m.n_tets);
  parallel_for(m.n_tets, [&](int64_t b, int64_t e) {
    for (int64_t t = b; t < e; ++t) {
      int32_t c = m.tet_cmpt[t];
      for (int a = 0; a < nv; ++a) {
        int32_t v = m.master[m.tets[nv * t + a]];
        int64_t d = base[v];
        while (m.dof_cmpt[d] != c) ++d;
        m.tet_dof[nv * t + a] = (int32_t)d;
      }
    }
  });
}

// Faces (edges in 2-D) shared by two elements of different compartments; a
// 1-D mesh has none, its nodes carrying one dof each.  Only faces whose
// three (master) vertices all carry more than one dof can be interface faces.
void find_interface_faces(HostMesh& m) {
  std::vector<uint8_t> multi(m.n_nodes, 0);
  for (int64_t d = 1; d < m.n_dof; ++d)
    if (m.dof_node[d] == m.dof_node[d - 1]) multi[m.dof_node[d]] = 1;
  // faces of a tetrahedron (vertex triples) or edges of a triangle (pairs)
  static const int LOC4[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  static const int LOC3[3][3] = {{1, 2, -1}, {0, 2, -1}, {0, 1, -1}};
  static const int LOC2[2][3] = {{1, -1, -1}, {0, -1, -1}};
  const int nv = m.nv, fs = nv - 1;
  auto LOC = [&](int f, int a) { return nv == 4 ? LOC4[f][a] : nv == 3 ? LOC3[f][a] : LOC2[f][a]; };
  struct Cand {
    std::array<int32_t, 3> key;
    int32_t tet;
    int8_t lf;
  };
  // candidates gathered by element chunks in parallel; the sort below orders
  // them by (key, element), which no gathering order can change
  std::mutex mu;
  std::vector<std::pair<int64_t, std::vector<Cand>>> parts;
  parallel_for(m.n_tets, [&](int64_t b, int64_t e) {
    std::vector<Cand> local;
    for (int64_t t = b; t < e; ++t) {
      for (int f = 0; f < nv; ++f) {
        std::array<int32_t, 3> k = {-1, -1, -1};
        bool ok = true;
        for (int a = 0; a < fs; ++a) {
          k[a] = m.master[m.tets[nv * t + LOC(f, a)]];
          ok = ok && multi[k[a]];
        }
        if (!ok) continue;
        std::sort(k.begin(), k.end());
        local.push_back({k, (int32_t)t, (int8_t)f});
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    parts.emplace_back(b, std::move(local));
  });
  std::sort(parts.begin(), parts.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<Cand> cand;
  for (auto& pt : parts) cand.insert(cand.end(), pt.second.begin(), pt.second.end());
  std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    return a.key != b.key ? a.key < b.key : a.tet < b.tet;
  });
  m.face_ta.clear();
  m.face_tb.clear();
  m.face_lv.clear();
  m.face_dof.clear();
  m.face_kappa.clear();
  for (size_t i = 0; i + 1 < cand.size(); ++i) {
    if (cand[i].key != cand[i + 1].key) continue;
    int32_t ta = cand[i].tet, tb = cand[i + 1].tet;
    int32_t ca = m.tet_cmpt[ta], cb = m.tet_cmpt[tb];
    if (ca == cb) continue;
    m.face_ta.push_back(ta);
    m.face_tb.push_back(tb);
    int32_t dofs[6];
    for (int a = 0; a < fs; ++a) {
      int la = LOC(cand[i].lf, a);
      m.face_lv.push_back((int8_t)la);
      dofs[a] = m.tet_dof[nv * ta + la];
      int32_t v = m.master[m.tets[nv * ta + la]];
      int lb = 0;
      while (m.master[m.tets[nv * tb + lb]] != v) ++lb;
      dofs[fs + a] = m.tet_dof[nv * tb + lb];
    }
    for (int a = 0; a < 2 * fs; ++a) m.face_dof.push_back(dofs[a]);
    double inv = 1.0 / m.kappa[ca] + 1.0 / m.kappa[cb];  // 1/inf = 0
    m.face_kappa.push_back(inv > 0 ? 1.0 / inv : INFINITY);
  }
  m.n_face = (int64_t)m.face_ta.size();
}

// Element and face incidence of every dof: the elements (faces) holding it,
// one entry per (element, local vertex) occurrence, in increasing element order.
struct Incidence {
  std::vector<int64_t> tp, fp;  // [n_dof + 1] offsets
  std::vector<int32_t> ti, fi;  // element (face) ids
};

Incidence build_incidence(const HostMesh& m) {
  const int64_t nd = m.n_dof, nt = m.n_tets, nf = m.n_face;
  const int nv = m.nv, nfd = 2 * (nv - 1);
  Incidence inc;
  inc.tp.assign(nd + 1, 0);
  inc.fp.assign(nd + 1, 0);
  for (int64_t i = 0; i < nv * nt; ++i) inc.tp[m.tet_dof[i] + 1]++;
  for (int64_t i = 0; i < nfd * nf; ++i) inc.fp[m.face_dof[i] + 1]++;
  for (int64_t d = 0; d < nd; ++d) {
    inc.tp[d + 1] += inc.tp[d];
    inc.fp[d + 1] += inc.fp[d];
  }
  inc.ti.resize(nv * nt);
  inc.fi.resize(nfd * nf);
  std::vector<int64_t> pos(inc.tp.begin(), inc.tp.end() - 1);
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < nv; ++a) inc.ti[pos[m.tet_dof[nv * t + a]]++] = (int32_t)t;
  std::vector<int64_t> pf(inc.fp.begin(), inc.fp.end() - 1);
  for (int64_t f = 0; f < nf; ++f)
    for (int a = 0; a < nfd; ++a) inc.fi[pf[m.face_dof[nfd * f + a]]++] = (int32_t)f;
  return inc;
}

void build_pattern(HostMesh& m, const Incidence& inc) {
  const int64_t nd = m.n_dof;
  const int nv = m.nv, nfd = 2 * (nv - 1);
  auto row_cols = [&](int64_t d, std::vector<int32_t>& buf) {
    buf.clear();
    for (int64_t k = inc.tp[d]; k < inc.tp[d + 1]; ++k)
      for (int a = 0; a < nv; ++a) buf.push_back(m.tet_dof[nv * (int64_t)inc.ti[k] + a]);
    for (int64_t k = inc.fp[d]; k < inc.fp[d + 1]; ++k)
      for (int a = 0; a < nfd; ++a) buf.push_back(m.face_dof[nfd * (int64_t)inc.fi[k] + a]);
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
  };
  std::vector<int64_t> len(nd);
  parallel_for(nd, [&](int64_t b, int64_t e) {
    std::vector<int32_t> buf;
    for (int64_t d = b; d < e; ++d) {
      row_cols(d, buf);
      len[d] = (int64_t)buf.size();
    }
  });
  m.row_ptr.assign(nd + 1, 0);
  for (int64_t d = 0; d < nd; ++d) m.row_ptr[d + 1] = m.row_ptr[d] + len[d];
  m.nnz = m.row_ptr[nd];
  m.col.resize(m.nnz);
  parallel_for(nd, [&](int64_t b, int64_t e) {
    std::vector<int32_t> buf;
    for (int64_t d = b; d < e; ++d) {
      row_cols(d, buf);
      std::copy(buf.begin(), buf.end(), m.col.begin() + m.row_ptr[d]);
    }
  });
}

// Slot-sorted contribution lists for one kind of entity (elements with w
// nodes, or interface faces with w dofs), built row by row in parallel: the
// slots of row d receive entries only from entities holding dof d.  Walking
// those in increasing entity order, and each entity's local rows and columns
// in increasing order, lists every slot's entries by increasing code
// w^2 entity + w a + b, so each slot sums its entries in a fixed order and the
// assembly is deterministic.  Row d's entries start at (occurrences before d) x w.
void slot_lists(const HostMesh& m, const std::vector<int64_t>& ip, const std::vector<int32_t>& ids,
                const std::vector<int32_t>& edof, int w, std::vector<int64_t>& cptr, std::vector<int32_t>& codes) {
  const int64_t nd = m.n_dof;
  cptr.assign(m.nnz + 1, 0);
  codes.resize(ip[nd] * w);
  cptr[m.nnz] = ip[nd] * w;
  parallel_for(nd, [&](int64_t b, int64_t e) {
    std::vector<int32_t> cnt, lslot, lcode;
    for (int64_t d = b; d < e; ++d) {
      const int64_t r0 = m.row_ptr[d], rl = m.row_ptr[d + 1] - r0;
      const int32_t* cols = m.col.data() + r0;
      cnt.assign(rl + 1, 0);
      lslot.clear();
      lcode.clear();
      for (int64_t k = ip[d]; k < ip[d + 1];) {
        const int32_t t = ids[k];
        while (k < ip[d + 1] && ids[k] == t) ++k;  // an entity holding d at several local vertices
        const int32_t* ed = &edof[(int64_t)w * t];
        for (int a = 0; a < w; ++a) {
          if (ed[a] != d) continue;
          for (int c = 0; c < w; ++c) {
            const int32_t s = (int32_t)(std::lower_bound(cols, cols + rl, ed[c]) - cols);
            lslot.push_back(s);
            lcode.push_back(w * w * t + w * a + c);
            cnt[s + 1]++;
          }
        }
      }
      for (int64_t s = 0; s < rl; ++s) cnt[s + 1] += cnt[s];
      const int64_t base = ip[d] * w;
      for (int64_t s = 0; s < rl; ++s) cptr[r0 + s] = base + cnt[s];
      for (size_t q = 0; q < lslot.size(); ++q) codes[base + cnt[lslot[q]]++] = lcode[q];
    }
  });
}

void build_contributions(HostMesh& m, const Incidence& inc) {
  const int nv = m.nv, nfd = 2 * (nv - 1);
  slot_lists(m, inc.tp, inc.ti, m.tet_dof, nv, m.tc_ptr, m.tc);
  slot_lists(m, inc.fp, inc.fi, m.face_dof, nfd, m.fc_ptr, m.fc);
}

}  // namespace

// 16-bit spread for a 48-bit Morton code
static uint64_t spread3(uint64_t v) {
  v &= 0xFFFFull;
  v = (v | (v << 16)) & 0x0000FF0000FFull;
  v = (v | (v << 8)) & 0x00F00F00F00Full;
  v = (v | (v << 4)) & 0x0C30C30C30C3ull;
  v = (v | (v << 2)) & 0x249249249249ull;
  return v;
}

void build_halo_tiles(const HostMesh& m, const std::vector<int64_t>& seg_row0, int umax, int tmax, int emax,
                      HaloTiles& t, bool sort_by_len) {
  t = HaloTiles();
  t.umax = umax;
  const int G = (int)seg_row0.size() - 1;
  const int64_t n = m.n_dof;
  t.rows.reserve(n);
  t.rowe.reserve(n + 1);
  t.rowl.reserve(n);
  t.lidx.reserve(m.nnz);
  t.slot.reserve(m.nnz);
  std::vector<int32_t> mark(n, -1);
  std::vector<std::pair<uint64_t, int32_t>> order;
  int32_t tid = 0;
  for (int g = 0; g < G; ++g) {
    t.seg_tile0.push_back((int32_t)t.r0.size());
    const int64_t a = seg_row0[g], b = seg_row0[g + 1];
    if (a == b) continue;
    // Morton order of the rows' node coordinates over the segment's bounding box
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t r = a; r < b; ++r)
      for (int k = 0; k < 3; ++k) {
        const double x = m.xyz[3 * (size_t)m.dof_node[r] + k];
        lo[k] = std::min(lo[k], x);
        hi[k] = std::max(hi[k], x);
      }
    order.clear();
    for (int64_t r = a; r < b; ++r) {
      uint64_t code = 0;
      for (int k = 0; k < 3; ++k) {
        const double ext = hi[k] - lo[k];
        const double f = ext > 0 ? (m.xyz[3 * (size_t)m.dof_node[r] + k] - lo[k]) / ext : 0.0;
        code |= spread3((uint64_t)std::min(65535.0, std::floor(f * 65535.0 + 0.5))) << k;
      }
      order.emplace_back(code, (int32_t)r);
    }
    std::sort(order.begin(), order.end());
    // greedy tiles along the curve: at most tmax rows, umax distinct columns
    // and emax entries.  The boundaries need one pass in order (a tile's
    // distinct columns depend on the rows before it); the tiles' halos, local
    // indices and entries are then written in parallel at their offsets.
    struct Span {
      size_t i0, i1;   // rows order[i0, i1)
      int32_t nu;      // distinct columns
      int64_t ne;      // entries
    };
    std::vector<Span> spans;
    size_t i = 0;
    while (i < order.size()) {
      Span sp{i, i, 0, 0};
      for (; i < order.size() && (int)(i - sp.i0) < tmax; ++i) {
        const int32_t r = order[i].second;
        const int64_t rn = m.row_ptr[r + 1] - m.row_ptr[r];
        int fresh = 0;
        for (int64_t k = m.row_ptr[r]; k < m.row_ptr[r + 1]; ++k) fresh += mark[m.col[k]] != tid;
        if (sp.nu + fresh > umax || sp.ne + rn > emax) {
          if (i == sp.i0) {
            // a single row wider than umax (or emax) cannot be staged
            t.too_wide = true;
            return;
          }
          break;
        }
        sp.ne += rn;
        sp.nu += fresh;
        for (int64_t k = m.row_ptr[r]; k < m.row_ptr[r + 1]; ++k) mark[m.col[k]] = tid;
      }
      sp.i1 = i;
      spans.push_back(sp);
      ++tid;
    }
    const size_t T0 = t.r0.size(), nrow0 = t.rows.size(), nu0 = t.ucol.size(), ne0 = t.lidx.size();
    std::vector<int64_t> ro(spans.size() + 1, 0), uo(spans.size() + 1, 0), eo(spans.size() + 1, 0);
    for (size_t s2 = 0; s2 < spans.size(); ++s2) {
      ro[s2 + 1] = ro[s2] + (int64_t)(spans[s2].i1 - spans[s2].i0);
      uo[s2 + 1] = uo[s2] + spans[s2].nu;
      eo[s2 + 1] = eo[s2] + spans[s2].ne;
    }
    t.r0.resize(T0 + spans.size());
    t.u0.resize(T0 + spans.size());
    t.e0.resize(T0 + spans.size());
    t.rows.resize(nrow0 + ro.back());
    t.rowe.resize(nrow0 + ro.back());
    t.rowl.resize(nrow0 + ro.back());
    t.ucol.resize(nu0 + uo.back());
    t.lidx.resize(ne0 + eo.back());
    t.slot.resize(ne0 + eo.back());
    std::atomic<bool> bad{false};
    parallel_for((int64_t)spans.size(), [&](int64_t b0, int64_t b1) {
      std::vector<int32_t> uc, span_rows;
      for (int64_t s2 = b0; s2 < b1; ++s2) {
        const Span& sp = spans[s2];
        uc.clear();
        for (size_t q = sp.i0; q < sp.i1; ++q) {
          const int32_t r = order[q].second;
          uc.insert(uc.end(), m.col.begin() + m.row_ptr[r], m.col.begin() + m.row_ptr[r + 1]);
        }
        std::sort(uc.begin(), uc.end());
        uc.erase(std::unique(uc.begin(), uc.end()), uc.end());
        if ((int32_t)uc.size() != sp.nu) {
          // the boundary pass counted a different number of distinct columns
          // (a row with a repeated column): the offsets would overlap
          bad.store(true);
          continue;
        }
        auto lp = [&](int32_t c) { return (int32_t)(std::lower_bound(uc.begin(), uc.end(), c) - uc.begin()); };
        t.r0[T0 + s2] = (int32_t)(nrow0 + ro[s2]);
        t.u0[T0 + s2] = (int32_t)(nu0 + uo[s2]);
        t.e0[T0 + s2] = (int32_t)(ne0 + eo[s2]);
        for (size_t u = 0; u < uc.size(); ++u) t.ucol[nu0 + uo[s2] + u] = (uint32_t)uc[u];
        int64_t e = ne0 + eo[s2];
        // owned rows in curve order, or longest first (rows of similar length
        // then share a warp in the slice-tiled apply)
        span_rows.clear();
        for (size_t q = sp.i0; q < sp.i1; ++q) span_rows.push_back(order[q].second);
        if (sort_by_len)
          std::stable_sort(span_rows.begin(), span_rows.end(), [&](int32_t x, int32_t y) {
            return m.row_ptr[x + 1] - m.row_ptr[x] > m.row_ptr[y + 1] - m.row_ptr[y];
          });
        for (size_t qq = 0; qq < span_rows.size(); ++qq) {
          const int32_t r = span_rows[qq];
          const size_t j = nrow0 + ro[s2] + qq;
          t.ucol[nu0 + uo[s2] + lp(r)] |= 0x80000000u;  // owned by this tile
          t.rows[j] = r;
          t.rowe[j] = (int32_t)e;
          t.rowl[j] = (uint16_t)lp(r);
          for (int64_t k = m.row_ptr[r]; k < m.row_ptr[r + 1]; ++k, ++e) {
            t.lidx[e] = (uint16_t)lp(m.col[k]);
            t.slot[e] = (int32_t)k;
          }
        }
      }
    });
    if (bad.load()) {
      t.too_wide = true;  // not stageable: the halo iteration is not offered
      return;
    }
  }
  t.seg_tile0.push_back((int32_t)t.r0.size());
  t.r0.push_back((int32_t)t.rows.size());
  t.u0.push_back((int32_t)t.ucol.size());
  t.e0.push_back((int32_t)t.lidx.size());
  t.rowe.push_back((int32_t)t.lidx.size());
}

int build_weak_periodic(const HostMesh& m, uint32_t axes, WeakPeriodic& wp, std::string& msg) {
  wp = WeakPeriodic();
  if (m.nv != 4 && m.nv != 3) {
    msg = "tetrahedral or triangular meshes only";
    return BT_EINVAL;
  }
  if (m.nv == 3 && (axes & 4u)) {
    msg = "a 2-D mesh couples the x and y sides only";
    return BT_EINVAL;
  }
  if (m.surface) {
    msg = "a surface has no box sides to couple";
    return BT_EINVAL;
  }
  const int nv = m.nv, fs = nv - 1;  // nodes per element, per boundary face
  double Lmax = 0, vsum = 0;
  for (int k = 0; k < 3; ++k) {
    wp.L[k] = m.hi[k] - m.lo[k];
    Lmax = std::max(Lmax, wp.L[k]);
  }
  const double tol = 1e-9 * Lmax;
  // boundary faces: vertex triples of a tetrahedron, vertex pairs of a triangle
  static const int LOC4[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  static const int LOC3[3][3] = {{1, 2, -1}, {0, 2, -1}, {0, 1, -1}};
  auto LOC = [&](int f, int a) { return nv == 4 ? LOC4[f][a] : LOC3[f][a]; };
  auto X = [&](int32_t v, int k) { return m.xyz[3 * (size_t)v + k]; };
  for (int64_t t = 0; t < m.n_tets; ++t) {
    const int32_t* tv = &m.tets[nv * t];
    double e[3][3];
    for (int a = 0; a < fs; ++a)
      for (int k = 0; k < 3; ++k) e[a][k] = X(tv[a + 1], k) - X(tv[0], k);
    if (nv == 4)
      vsum += std::fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                        e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                        e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) / 6.0;
    else
      vsum += 0.5 * std::fabs(e[0][0] * e[1][1] - e[0][1] * e[1][0]);
  }
  // the Kuhn cell edge: (d! x mean element measure)^(1/d)
  wp.h = nv == 4 ? std::cbrt(6.0 * vsum / (double)m.n_tets) : std::sqrt(2.0 * vsum / (double)m.n_tets);
  wp.B.assign(m.nnz, 0.0);
  auto slot = [&](int32_t r, int32_t c) -> int64_t {
    const int32_t* b = &m.col[m.row_ptr[r]];
    const int32_t* e = &m.col[m.row_ptr[r + 1]];
    const int32_t* it = std::lower_bound(b, e, c);
    return (it != e && *it == c) ? m.row_ptr[r] + (it - b) : -1;
  };
  // P1 mass of a face: measure / (fs (fs + 1)) (1 + delta_ab)
  auto face_measure = [&](const double P[3][3]) {
    const double u1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    if (fs == 2) return std::sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    const double u2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const double cx = u1[1] * u2[2] - u1[2] * u2[1], cy = u1[2] * u2[0] - u1[0] * u2[2],
                 cz = u1[0] * u2[1] - u1[1] * u2[0];
    return 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
  };
  const double mdiv = (double)(fs * (fs + 1));
  struct Face {
    int64_t t;
    int lf;
  };
  using Entry = std::tuple<int32_t, int32_t, double, int8_t>;  // row, col, w, code
  std::vector<Entry> ent;
  // The projection for sides that do not match: a node's partner value is the
  // opposite side's P1 field at the node shifted by +-L_k, read from the face
  // that contains the shifted point with its barycentric weights.  A uniform
  // grid over the side's tangential coordinates finds the candidate faces.
  auto project_axis = [&](int k, const std::vector<Face>* sides, std::vector<Entry>& out,
                          std::string& err) -> int {
    int ta[2] = {0, 0}, ntan = 0;  // tangential axes
    if (nv == 3) {
      ta[ntan++] = k == 0 ? 1 : 0;
    } else {
      for (int a = 0; a < 3; ++a)
        if (a != k) ta[ntan++] = a;
    }
    struct Rec {
      int32_t node[3], dof[3];
      double meas;
    };
    std::vector<Rec> rec[2];
    for (int sd = 0; sd < 2; ++sd)
      for (const Face& f : sides[sd]) {
        Rec r{};
        double P[3][3] = {};
        for (int a = 0; a < fs; ++a) {
          r.node[a] = m.tets[nv * f.t + LOC(f.lf, a)];
          r.dof[a] = m.tet_dof[nv * f.t + LOC(f.lf, a)];
          for (int kk = 0; kk < 3; ++kk) P[a][kk] = X(r.node[a], kk);
        }
        r.meas = face_measure(P);
        rec[sd].push_back(r);
      }
    // grids over each side's tangential box
    struct Grid {
      double lo[2] = {0, 0}, cell[2] = {1, 1};
      int n[2] = {1, 1};
      std::vector<std::vector<int32_t>> bins;
    } grid[2];
    for (int sd = 0; sd < 2; ++sd) {
      Grid& g = grid[sd];
      double hi[2] = {-1e300, -1e300};
      g.lo[0] = g.lo[1] = 1e300;
      for (const Rec& r : rec[sd])
        for (int a = 0; a < fs; ++a)
          for (int j = 0; j < ntan; ++j) {
            g.lo[j] = std::min(g.lo[j], X(r.node[a], ta[j]));
            hi[j] = std::max(hi[j], X(r.node[a], ta[j]));
          }
      const double per = ntan == 2 ? std::sqrt((double)rec[sd].size()) : (double)rec[sd].size();
      for (int j = 0; j < ntan; ++j) {
        g.n[j] = std::max(1, (int)std::min(4096.0, per));
        g.cell[j] = std::max((hi[j] - g.lo[j]) / g.n[j], 1e-300);
      }
      g.bins.assign((size_t)g.n[0] * g.n[1], {});
      for (size_t i = 0; i < rec[sd].size(); ++i) {
        int c0[2] = {0, 0}, c1[2] = {0, 0};
        for (int j = 0; j < ntan; ++j) {
          double a0 = 1e300, a1 = -1e300;
          for (int a = 0; a < fs; ++a) {
            a0 = std::min(a0, X(rec[sd][i].node[a], ta[j]));
            a1 = std::max(a1, X(rec[sd][i].node[a], ta[j]));
          }
          c0[j] = std::max(0, std::min(g.n[j] - 1, (int)std::floor((a0 - g.lo[j]) / g.cell[j])));
          c1[j] = std::max(0, std::min(g.n[j] - 1, (int)std::floor((a1 - g.lo[j]) / g.cell[j])));
        }
        for (int u = c0[0]; u <= c1[0]; ++u)
          for (int v = c0[1]; v <= c1[1]; ++v) g.bins[(size_t)u * g.n[1] + v].push_back((int32_t)i);
      }
    }
    // barycentric weights of the point y in face i of side sd (tangential coordinates)
    auto weights = [&](int sd, int32_t i, const double* y, double* lam) {
      const Rec& r = rec[sd][i];
      if (ntan == 1) {
        const double p0 = X(r.node[0], ta[0]), p1 = X(r.node[1], ta[0]);
        const double t = (y[ta[0]] - p0) / (p1 - p0);
        lam[0] = 1.0 - t;
        lam[1] = t;
        return;
      }
      const double u0 = X(r.node[0], ta[0]), v0 = X(r.node[0], ta[1]);
      const double e1u = X(r.node[1], ta[0]) - u0, e1v = X(r.node[1], ta[1]) - v0;
      const double e2u = X(r.node[2], ta[0]) - u0, e2v = X(r.node[2], ta[1]) - v0;
      const double du = y[ta[0]] - u0, dv = y[ta[1]] - v0;
      const double det = e1u * e2v - e1v * e2u;
      lam[1] = (du * e2v - dv * e2u) / det;
      lam[2] = (e1u * dv - e1v * du) / det;
      lam[0] = 1.0 - lam[1] - lam[2];
    };
    auto locate = [&](int sd, const double* y, int32_t* pd, double* pw) -> bool {
      const Grid& g = grid[sd];
      int c[2] = {0, 0};
      for (int j = 0; j < ntan; ++j)
        c[j] = std::max(0, std::min(g.n[j] - 1, (int)std::floor((y[ta[j]] - g.lo[j]) / g.cell[j])));
      double best = -1e300, lam[3];
      int32_t bi = -1;
      auto consider = [&](int32_t i) {
        weights(sd, i, y, lam);
        double mn = lam[0];
        for (int a = 1; a < fs; ++a) mn = std::min(mn, lam[a]);
        if (mn > best) {
          best = mn;
          bi = i;
        }
      };
      for (int32_t i : g.bins[(size_t)c[0] * g.n[1] + c[1]]) consider(i);
      if (best < -1e-9)  // not in its cell's candidates: search the whole side
        for (int32_t i = 0; i < (int32_t)rec[sd].size(); ++i) consider(i);
      if (bi < 0 || best < -1e-9) return false;
      weights(sd, bi, y, lam);
      for (int a = 0; a < fs; ++a) {
        pd[a] = rec[sd][bi].dof[a];
        pw[a] = lam[a];
      }
      return true;
    };
    for (int sd = 0; sd < 2; ++sd) {
      const int other = 1 - sd;
      const double shift = sd == 0 ? wp.L[k] : -wp.L[k];
      std::map<int32_t, std::pair<std::array<int32_t, 3>, std::array<double, 3>>> partner;
      for (const Rec& r : rec[sd]) {
        for (int b = 0; b < fs; ++b) {
          if (partner.count(r.node[b])) continue;
          double y[3] = {X(r.node[b], 0), X(r.node[b], 1), X(r.node[b], 2)};
          y[k] += shift;
          std::array<int32_t, 3> pd = {-1, -1, -1};
          std::array<double, 3> pw = {0, 0, 0};
          if (!locate(other, y, pd.data(), pw.data())) {
            err = "a node's partner point lies outside the opposite side on axis " + std::to_string(k);
            return BT_EINVAL;
          }
          for (int a = 0; a < fs; ++a)
            if (pd[a] < 0 || pd[a] >= m.n_dof) {
              err = "partner face lookup failed on axis " + std::to_string(k);
              return BT_EINVAL;
            }
          partner[r.node[b]] = {pd, pw};
        }
        for (int a = 0; a < fs; ++a)
          for (int b = 0; b < fs; ++b) {
            const double wt = r.meas / mdiv * (a == b ? 2.0 : 1.0);
            const auto& pr = partner[r.node[b]];
            for (int c = 0; c < fs; ++c)
              if (pr.second[c] != 0.0)
                out.emplace_back(r.dof[a], pr.first[c], wt * pr.second[c], (int8_t)(sd ? (k | 4) : k));
          }
      }
    }
    return BT_OK;
  };
  for (int k = 0; k < 3; ++k) {
    if (!((axes >> k) & 1)) continue;
    std::vector<Face> side[2];
    for (int64_t t = 0; t < m.n_tets; ++t)
      for (int f = 0; f < nv; ++f)
        for (int sd = 0; sd < 2; ++sd) {
          const double plane = sd ? m.hi[k] : m.lo[k];
          bool on = true;
          for (int a = 0; a < fs; ++a) on &= std::fabs(X(m.tets[nv * t + LOC(f, a)], k) - plane) < tol;
          if (on) side[sd].push_back({t, f});
        }
    // slave faces by their sorted node ids (-1 pads an edge); slave nodes by coordinates
    std::map<std::array<int32_t, 3>, Face> sface;
    std::map<std::array<int64_t, 3>, int32_t> snode;
    auto qkey = [&](double x, double y, double z) {
      return std::array<int64_t, 3>{(int64_t)std::llround(x / tol), (int64_t)std::llround(y / tol),
                                    (int64_t)std::llround(z / tol)};
    };
    for (const Face& f : side[1]) {
      std::array<int32_t, 3> key = {-1, -1, -1};
      for (int a = 0; a < fs; ++a) {
        key[a] = m.tets[nv * f.t + LOC(f.lf, a)];
        snode[qkey(X(key[a], 0), X(key[a], 1), X(key[a], 2))] = key[a];
      }
      std::sort(key.begin(), key.end());
      sface[key] = f;
    }
    // matching sides: each master node's partner is the slave node at x + L_k e_k;
    // otherwise the projection below couples the sides
    bool matched = true;
    std::vector<std::tuple<int32_t, int32_t, double, int8_t>> axis_ent;
    for (int sd = 0; sd < 2; ++sd)
      for (const Face& f : side[sd]) {
        int32_t v[3], dof[3];
        double P[3][3] = {};
        for (int a = 0; a < fs; ++a) {
          v[a] = m.tets[nv * f.t + LOC(f.lf, a)];
          dof[a] = m.tet_dof[nv * f.t + LOC(f.lf, a)];
          for (int kk = 0; kk < 3; ++kk) P[a][kk] = X(v[a], kk);
        }
        const double meas = face_measure(P);
        for (int a = 0; a < fs; ++a)
          for (int b = 0; b < fs; ++b) {
            const int64_t sl = slot(dof[a], dof[b]);
            if (sl < 0) {
              msg = "boundary face entry outside the pattern";
              return BT_EINVAL;
            }
            wp.B[sl] += meas / mdiv * (a == b ? 2.0 : 1.0);
          }
        if (sd == 1 || !matched) continue;
        // master face: partner nodes at x + L_k e_k and the slave face holding them
        int32_t pv[3];
        std::array<int32_t, 3> key = {-1, -1, -1};
        bool all = true;
        for (int a = 0; a < fs && all; ++a) {
          double y[3] = {P[a][0], P[a][1], P[a][2]};
          y[k] += wp.L[k];
          auto it = snode.find(qkey(y[0], y[1], y[2]));
          if (it == snode.end()) {
            all = false;
          } else {
            pv[a] = key[a] = it->second;
          }
        }
        std::sort(key.begin(), key.end());
        auto fit = all ? sface.find(key) : sface.end();
        if (fit == sface.end()) {
          matched = false;
          continue;
        }
        const Face& g = fit->second;
        int32_t pdof[3] = {-1, -1, -1};
        for (int a = 0; a < fs; ++a)
          for (int c = 0; c < fs; ++c)
            if (m.tets[nv * g.t + LOC(g.lf, c)] == pv[a]) pdof[a] = m.tet_dof[nv * g.t + LOC(g.lf, c)];
        for (int a = 0; a < fs; ++a)
          if (pdof[a] < 0 || pdof[a] >= m.n_dof) {
            msg = "partner face lookup failed on axis " + std::to_string(k);
            return BT_EINVAL;
          }
        for (int a = 0; a < fs; ++a)
          for (int b = 0; b < fs; ++b) {
            const double wt = meas / mdiv * (a == b ? 2.0 : 1.0);
            axis_ent.emplace_back(dof[a], pdof[b], wt, (int8_t)k);        // master row: slave value, +phase
            axis_ent.emplace_back(pdof[a], dof[b], wt, (int8_t)(k | 4));  // slave row: master value, -phase
          }
      }
    if (matched) {
      ent.insert(ent.end(), axis_ent.begin(), axis_ent.end());
    } else if (int st = project_axis(k, side, ent, msg)) {
      return st;
    }
  }
  std::stable_sort(ent.begin(), ent.end(),
                   [](const auto& x, const auto& y) { return std::get<0>(x) < std::get<0>(y); });
  for (size_t i = 0; i < ent.size(); ++i) {
    const int32_t r = std::get<0>(ent[i]);
    if (wp.rows.empty() || wp.rows.back() != r) {
      wp.rows.push_back(r);
      wp.ptr.push_back((int32_t)i);
    }
    wp.col.push_back(std::get<1>(ent[i]));
    wp.w.push_back(std::get<2>(ent[i]));
    wp.code.push_back(std::get<3>(ent[i]));
  }
  wp.ptr.push_back((int32_t)ent.size());
  return BT_OK;
}

int build_host_mesh(HostMesh& m, std::string& msg) {
  int st = validate(m, msg);
  if (st) return st;
  st = periodic_identify(m, msg);
  if (st) return st;
  double_interface_nodes(m);
  if (m.nv == 2)  // a manifold carries no membranes: one compartment per node
    for (int64_t d = 1; d < m.n_dof; ++d)
      if (m.dof_node[d] == m.dof_node[d - 1]) {
        msg = "segments of different compartments share node " + std::to_string(m.dof_node[d]);
        return BT_EINVAL;
      }
  find_interface_faces(m);
  if (m.nnz >= (int64_t(1) << 31)) {
    msg = "pattern too large";
    return BT_EINVAL;
  }
  const Incidence inc = build_incidence(m);
  build_pattern(m, inc);
  if (m.nnz >= (int64_t(1) << 31) || 36 * m.n_face >= (int64_t(1) << 31)) {
    msg = "pattern too large for 32-bit indexing";
    return BT_EINVAL;
  }
  build_contributions(m, inc);
  return BT_OK;
}

}  // namespace bt
