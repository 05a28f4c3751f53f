// Mesh structure on the host: node coordinates, cells, the column-offset set of
// the pattern, per-row presence masks and node-to-cell incidence.  Integer and
// coordinate bookkeeping only; every matrix entry is computed on the device.
#include <algorithm>
#include <cstring>
#include <map>

#include "afc_internal.h"

namespace afc {

namespace {

// Kuhn split of a box cell: for the axis order (a, b, c), the tetrahedron
// {0, e_a, e_a + e_b, e_a + e_b + e_c} in local corner numbering dx + 2dy + 4dz.
void kuhn_tets(int tets[6][4]) {
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int t = 0; t < 6; ++t) {
    int a = perm[t][0], b = perm[t][1];
    tets[t][0] = 0;
    tets[t][1] = 1 << a;
    tets[t][2] = (1 << a) | (1 << b);
    tets[t][3] = 7;
  }
}

int finish_structure(MeshStructure& m, const std::vector<int32_t>& offsets) {
  if ((int)offsets.size() > kMaxOffsets) {
    set_error("mesh pattern has " + std::to_string(offsets.size()) + " column offsets (max " +
              std::to_string(kMaxOffsets) + ")");
    return AFC_E_INVALID;
  }
  m.offsets = offsets;
  // incidence by counting sort
  const int64_t N = m.N;
  m.inc_ptr.assign(N + 1, 0);
  for (int64_t e = 0; e < m.ncells; ++e)
    for (int a = 0; a < m.nl; ++a) m.inc_ptr[m.conn[e * m.nl + a] + 1]++;
  for (int64_t i = 0; i < N; ++i) m.inc_ptr[i + 1] += m.inc_ptr[i];
  m.inc.assign((size_t)m.inc_ptr[N], 0);
  std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
  for (int64_t e = 0; e < m.ncells; ++e)
    for (int a = 0; a < m.nl; ++a) {
      int32_t i = m.conn[e * m.nl + a];
      m.inc[fill[i]++] = (int32_t)((e << 3) | a);
    }
  int64_t nnz = 0;
  for (int64_t i = 0; i < N; ++i) nnz += __builtin_popcountll(m.mask[i]);
  m.nnz = nnz;
  m.n_edges = (nnz - N) / 2;
  return AFC_OK;
}

}  // namespace

int build_structured(int elem, int nx, int ny, int nz, const double lo[3], const double hi[3], MeshStructure& m) {
  if (elem != AFC_P1 && elem != AFC_Q1) { set_error("elem must be AFC_P1 or AFC_Q1"); return AFC_E_INVALID; }
  if (nx < 2 || ny < 2 || nz < 2) { set_error("need at least 2 nodes per side"); return AFC_E_INVALID; }
  const int64_t N = (int64_t)nx * ny * nz;
  if (N > (int64_t)1 << 30) { set_error("too many nodes"); return AFC_E_INVALID; }
  for (int d = 0; d < 3; ++d)
    if (!(hi[d] > lo[d])) { set_error("box must have hi > lo"); return AFC_E_INVALID; }
  m = MeshStructure();
  m.elem = elem;
  m.nl = elem == AFC_P1 ? 4 : 8;
  m.N = N;
  m.xyz.resize(3 * N);
  const int n[3] = {nx, ny, nz};
  for (int64_t iz = 0; iz < nz; ++iz)
    for (int64_t iy = 0; iy < ny; ++iy)
      for (int64_t ix = 0; ix < nx; ++ix) {
        int64_t i = ix + nx * (iy + ny * iz);
        const int64_t id[3] = {ix, iy, iz};
        for (int d = 0; d < 3; ++d) {
          // node placement of a linspace: k * (hi - lo) / (n - 1) + lo, last node at hi
          double step = (hi[d] - lo[d]) / (double)(n[d] - 1);
          m.xyz[3 * i + d] = id[d] == n[d] - 1 ? hi[d] : (double)id[d] * step + lo[d];
        }
      }
  const int64_t cells = (int64_t)(nx - 1) * (ny - 1) * (nz - 1);
  int32_t corner_off[8];
  for (int k = 0; k < 8; ++k) corner_off[k] = (k & 1) + nx * (((k >> 1) & 1) + ny * ((k >> 2) & 1));
  int tets[6][4];
  kuhn_tets(tets);
  const int per_cube = elem == AFC_P1 ? 6 : 1;
  m.ncells = cells * per_cube;
  m.conn.resize((size_t)(m.ncells * m.nl));
  // local vertex lists of the cell types
  std::vector<std::vector<int>> types;
  if (elem == AFC_P1)
    for (int t = 0; t < 6; ++t) types.push_back({tets[t][0], tets[t][1], tets[t][2], tets[t][3]});
  else
    types.push_back({0, 1, 2, 3, 4, 5, 6, 7});
  // offsets of the pattern: differences of corner offsets within each type
  std::vector<int32_t> offs;
  for (auto& ty : types)
    for (int a : ty)
      for (int b : ty) offs.push_back(corner_off[b] - corner_off[a]);
  std::sort(offs.begin(), offs.end());
  offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
  auto kof = [&](int32_t o) { return (int)(std::lower_bound(offs.begin(), offs.end(), o) - offs.begin()); };
  std::vector<std::vector<std::vector<int>>> kpair(types.size());
  for (size_t t = 0; t < types.size(); ++t) {
    int nl = (int)types[t].size();
    kpair[t].assign(nl, std::vector<int>(nl));
    for (int a = 0; a < nl; ++a)
      for (int b = 0; b < nl; ++b) kpair[t][a][b] = kof(corner_off[types[t][b]] - corner_off[types[t][a]]);
  }
  m.mask.assign(N, 0ull);
  int64_t e = 0;
  for (int t = 0; t < per_cube; ++t) {
    for (int64_t cz = 0; cz < nz - 1; ++cz)
      for (int64_t cy = 0; cy < ny - 1; ++cy)
        for (int64_t cx = 0; cx < nx - 1; ++cx, ++e) {
          int32_t base = (int32_t)(cx + nx * (cy + ny * cz));
          const auto& ty = types[t];
          for (int a = 0; a < m.nl; ++a) m.conn[e * m.nl + a] = base + corner_off[ty[a]];
          for (int a = 0; a < m.nl; ++a) {
            uint64_t bits = 0;
            for (int b = 0; b < m.nl; ++b) bits |= 1ull << kpair[t][a][b];
            m.mask[base + corner_off[ty[a]]] |= bits;
          }
        }
  }
  return finish_structure(m, offs);
}

int build_from_elements(int elem, int64_t n_nodes, const double* xyz, int64_t n_cells, const int32_t* conn,
                        MeshStructure& m) {
  if (elem != AFC_P1 && elem != AFC_Q1) { set_error("elem must be AFC_P1 or AFC_Q1"); return AFC_E_INVALID; }
  if (n_nodes < 2 || n_cells < 1 || !xyz || !conn) { set_error("empty mesh"); return AFC_E_INVALID; }
  if (n_nodes > (int64_t)1 << 30 || n_cells > (int64_t)1 << 28) { set_error("mesh too large"); return AFC_E_INVALID; }
  m = MeshStructure();
  m.elem = elem;
  m.nl = elem == AFC_P1 ? 4 : 8;
  m.N = n_nodes;
  m.ncells = n_cells;
  m.xyz.assign(xyz, xyz + 3 * n_nodes);
  m.conn.assign(conn, conn + m.nl * n_cells);
  for (int64_t e = 0; e < n_cells; ++e) {
    for (int a = 0; a < m.nl; ++a) {
      int32_t v = m.conn[e * m.nl + a];
      if (v < 0 || v >= n_nodes) { set_error("connectivity index out of range"); return AFC_E_INVALID; }
      for (int b = 0; b < a; ++b)
        if (m.conn[e * m.nl + b] == v) { set_error("repeated vertex in a cell"); return AFC_E_INVALID; }
    }
  }
  std::map<int32_t, int> seen;
  for (int64_t e = 0; e < n_cells; ++e)
    for (int a = 0; a < m.nl; ++a)
      for (int b = 0; b < m.nl; ++b) seen[m.conn[e * m.nl + b] - m.conn[e * m.nl + a]] = 0;
  // the offset set must be symmetric and contain 0 by construction
  std::vector<int32_t> offs;
  for (auto& kv : seen) offs.push_back(kv.first);
  if ((int)offs.size() > kMaxOffsets) {
    set_error("mesh pattern has " + std::to_string(offs.size()) + " column offsets (max " +
              std::to_string(kMaxOffsets) + "); renumber the nodes");
    return AFC_E_INVALID;
  }
  for (size_t k = 0; k < offs.size(); ++k) seen[offs[k]] = (int)k;
  m.mask.assign(n_nodes, 0ull);
  for (int64_t e = 0; e < n_cells; ++e)
    for (int a = 0; a < m.nl; ++a)
      for (int b = 0; b < m.nl; ++b) {
        int32_t i = m.conn[e * m.nl + a], j = m.conn[e * m.nl + b];
        m.mask[i] |= 1ull << seen[j - i];
      }
  return finish_structure(m, offs);
}

}  // namespace afc
