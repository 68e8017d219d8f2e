// lim_codes.cpp -- host construction of codes: CSR validation, the CSC view of
// the Tanner graph (Sec. S1), the CSS condition H_Z H_X^T = 0 (Preliminaries),
// X-logicals (a basis of ker H_Z modulo row H_X, decoding criterion (2)) and the
// code families simulated in the paper.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lim_internal.h"

namespace lim {

namespace {

int fail(int st, const std::string &msg) {
  set_error(msg);
  return st;
}

// A GF(2) row from a list of columns: sorted, repeated columns cancel.
std::vector<int32_t> gf2_row(std::vector<int32_t> cols) {
  std::sort(cols.begin(), cols.end());
  std::vector<int32_t> out;
  for (size_t i = 0; i < cols.size();) {
    size_t j = i;
    while (j < cols.size() && cols[j] == cols[i]) j++;
    if ((j - i) & 1) out.push_back(cols[i]);
    i = j;
  }
  return out;
}

void to_csr(const std::vector<std::vector<int32_t>> &rows, std::vector<int32_t> &ptr,
            std::vector<int32_t> &col) {
  ptr.assign(1, 0);
  col.clear();
  for (auto &r : rows) {
    col.insert(col.end(), r.begin(), r.end());
    ptr.push_back((int32_t)col.size());
  }
}

// Dense bit vector helpers for GF(2) elimination (small codes only).
using BitVec = std::vector<uint64_t>;

int highest_bit(const BitVec &v) {
  for (int w = (int)v.size() - 1; w >= 0; w--)
    if (v[w]) return w * 64 + 63 - __builtin_clzll(v[w]);
  return -1;
}

void xor_into(BitVec &a, const BitVec &b) {
  for (size_t i = 0; i < a.size(); i++) a[i] ^= b[i];
}

// Reduces x against a basis keyed by leading bit; returns true if x became 0.
bool reduce(BitVec &x, const std::map<int, BitVec> &basis) {
  for (;;) {
    int hb = highest_bit(x);
    if (hb < 0) return true;
    auto it = basis.find(hb);
    if (it == basis.end()) return false;
    xor_into(x, it->second);
  }
}

// Basis of ker(H) for H given as CSR rows over n columns.
std::vector<BitVec> kernel_basis(int n, const std::vector<int32_t> &ptr,
                                 const std::vector<int32_t> &col) {
  int W = (n + 63) / 64;
  int rows = (int)ptr.size() - 1;
  std::vector<BitVec> a(rows, BitVec(W, 0));
  for (int r = 0; r < rows; r++)
    for (int j = ptr[r]; j < ptr[r + 1]; j++) a[r][col[j] / 64] ^= 1ull << (col[j] % 64);
  std::vector<int> pivot_col;
  int rank = 0;
  for (int c = 0; c < n && rank < rows; c++) {
    int piv = -1;
    for (int r = rank; r < rows; r++)
      if ((a[r][c / 64] >> (c % 64)) & 1) { piv = r; break; }
    if (piv < 0) continue;
    std::swap(a[piv], a[rank]);
    for (int r = 0; r < rows; r++)
      if (r != rank && ((a[r][c / 64] >> (c % 64)) & 1)) xor_into(a[r], a[rank]);
    pivot_col.push_back(c);
    rank++;
  }
  std::vector<char> is_piv(n, 0);
  for (int c : pivot_col) is_piv[c] = 1;
  std::vector<BitVec> out;
  for (int f = 0; f < n; f++) {
    if (is_piv[f]) continue;
    BitVec x(W, 0);
    x[f / 64] |= 1ull << (f % 64);
    for (int i = 0; i < rank; i++)
      if ((a[i][f / 64] >> (f % 64)) & 1) x[pivot_col[i] / 64] |= 1ull << (pivot_col[i] % 64);
    out.push_back(x);
  }
  return out;
}

int logicals_from_hz(int n, const std::vector<int32_t> &hx_ptr, const std::vector<int32_t> &hx_col,
                     const std::vector<int32_t> &hz_ptr, const std::vector<int32_t> &hz_col,
                     std::vector<uint32_t> &logicals, int32_t &k) {
  if (n > 4096)
    return fail(LIM_E_UNSUPPORTED, "automatic logicals need n <= 4096; pass them explicitly");
  int W = (n + 63) / 64;
  std::map<int, BitVec> span;
  int mx = (int)hx_ptr.size() - 1;
  for (int r = 0; r < mx; r++) {
    BitVec x(W, 0);
    for (int j = hx_ptr[r]; j < hx_ptr[r + 1]; j++) x[hx_col[j] / 64] ^= 1ull << (hx_col[j] % 64);
    if (!reduce(x, span)) span[highest_bit(x)] = x;
  }
  std::vector<BitVec> ker;
  if (hz_ptr.size() > 1) {
    ker = kernel_basis(n, hz_ptr, hz_col);
  } else {
    for (int v = 0; v < n; v++) {
      BitVec x(W, 0);
      x[v / 64] |= 1ull << (v % 64);
      ker.push_back(x);
    }
  }
  std::vector<BitVec> lg;
  for (auto &x0 : ker) {
    BitVec x = x0;
    if (!reduce(x, span)) {
      span[highest_bit(x)] = x;
      lg.push_back(x0);
    }
  }
  if ((int)lg.size() > LIM_MAX_LOGICALS)
    return fail(LIM_E_UNSUPPORTED, "more than LIM_MAX_LOGICALS logical operators");
  k = (int32_t)lg.size();
  int nw = (n + 31) / 32;
  logicals.assign((size_t)k * nw, 0);
  for (int j = 0; j < k; j++)
    for (int v = 0; v < n; v++)
      if ((lg[j][v / 64] >> (v % 64)) & 1) logicals[(size_t)j * nw + v / 32] |= 1u << (v % 32);
  return LIM_OK;
}

// CSC view and degrees; assumes a validated CSR.
void finish(HostCode &hc) {
  int n = hc.n, m = hc.m;
  hc.E = hc.c_ptr[m];
  hc.v_ptr.assign(n + 1, 0);
  for (int e = 0; e < hc.E; e++) hc.v_ptr[hc.c_var[e] + 1]++;
  for (int v = 0; v < n; v++) hc.v_ptr[v + 1] += hc.v_ptr[v];
  hc.v_edge.assign(hc.E, 0);
  hc.v_chk.assign(hc.E, 0);
  std::vector<int32_t> fill(n, 0);
  for (int c = 0; c < m; c++)  // ascending c: each qubit's list is ascending in c
    for (int e = hc.c_ptr[c]; e < hc.c_ptr[c + 1]; e++) {
      int v = hc.c_var[e];
      int pos = hc.v_ptr[v] + fill[v]++;
      hc.v_edge[pos] = e;
      hc.v_chk[pos] = c;
    }
  hc.dc_min = hc.dv_min = 1 << 30;
  hc.dc_max = hc.dv_max = 0;
  for (int c = 0; c < m; c++) {
    int d = hc.c_ptr[c + 1] - hc.c_ptr[c];
    hc.dc_min = std::min(hc.dc_min, d);
    hc.dc_max = std::max(hc.dc_max, d);
  }
  for (int v = 0; v < n; v++) {
    int d = hc.v_ptr[v + 1] - hc.v_ptr[v];
    hc.dv_min = std::min(hc.dv_min, d);
    hc.dv_max = std::max(hc.dv_max, d);
  }
  if (m == 0) hc.dc_min = 0;
  // For uniform degrees: for every edge (c, v), the other edges of v in
  // ascending check order -- the terms of v's message to c in Eq. 1.
  hc.partner.clear();
  if (hc.dv_min == hc.dv_max && hc.dv_max >= 2 && hc.dc_min == hc.dc_max && hc.dc_max >= 2) {
    const int dv = hc.dv_max;
    hc.partner.assign((size_t)hc.E * (dv - 1), 0);
    for (int v = 0; v < n; v++)
      for (int j = 0; j < dv; j++) {
        const int e = hc.v_edge[hc.v_ptr[v] + j];
        int o = 0;
        for (int jj = 0; jj < dv; jj++)
          if (jj != j) hc.partner[(size_t)e * (dv - 1) + o++] = hc.v_edge[hc.v_ptr[v] + jj];
      }
  }
}

int validate_csr(int32_t rows, int32_t n, const int32_t *ptr, const int32_t *col, const char *what) {
  if (rows < 0 || (rows > 0 && (!ptr || !col))) return fail(LIM_E_INVAL, std::string(what) + ": null CSR");
  if (rows == 0) return LIM_OK;
  if (ptr[0] != 0) return fail(LIM_E_INVAL, std::string(what) + ": row pointer must start at 0");
  for (int r = 0; r < rows; r++) {
    if (ptr[r + 1] < ptr[r]) return fail(LIM_E_INVAL, std::string(what) + ": row pointer decreases");
    for (int j = ptr[r]; j < ptr[r + 1]; j++) {
      if (col[j] < 0 || col[j] >= n) return fail(LIM_E_INVAL, std::string(what) + ": column out of range");
      if (j > ptr[r] && col[j - 1] >= col[j])
        return fail(LIM_E_INVAL, std::string(what) + ": columns must be strictly ascending");
    }
  }
  return LIM_OK;
}

int assemble(int32_t n, const std::vector<std::vector<int32_t>> &hx_rows,
             const std::vector<std::vector<int32_t>> *hz_rows,
             const std::vector<std::vector<int32_t>> *logical_sets, HostCode &out) {
  std::vector<int32_t> hp, hc, zp, zc;
  to_csr(hx_rows, hp, hc);
  if (hz_rows) to_csr(*hz_rows, zp, zc);
  std::vector<uint32_t> lg;
  int32_t k = 0;
  if (logical_sets) {
    int nw = (n + 31) / 32;
    k = (int32_t)logical_sets->size();
    lg.assign((size_t)k * nw, 0);
    for (int j = 0; j < k; j++)
      for (int v : (*logical_sets)[j]) lg[(size_t)j * nw + v / 32] ^= 1u << (v % 32);
  }
  return build_from_csr((int32_t)hx_rows.size(), n, hp.data(), hc.data(),
                        hz_rows ? (int32_t)hz_rows->size() : 0, hz_rows ? zp.data() : nullptr,
                        hz_rows ? zc.data() : nullptr, k, logical_sets ? lg.data() : nullptr, out);
}

}  // namespace

int build_from_csr(int32_t m, int32_t n, const int32_t *hx_ptr, const int32_t *hx_col, int32_t mz,
                   const int32_t *hz_ptr, const int32_t *hz_col, int32_t k,
                   const uint32_t *logicals, HostCode &out) {
  if (n <= 0 || m <= 0) return fail(LIM_E_INVAL, "code needs n > 0 and m > 0");
  int st = validate_csr(m, n, hx_ptr, hx_col, "H_X");
  if (st) return st;
  if (mz > 0) {
    st = validate_csr(mz, n, hz_ptr, hz_col, "H_Z");
    if (st) return st;
  }
  out = HostCode();
  out.n = n;
  out.m = m;
  out.c_ptr.assign(hx_ptr, hx_ptr + m + 1);
  out.c_var.assign(hx_col, hx_col + hx_ptr[m]);
  finish(out);
  if (out.dc_max > kMaxDeg || out.dv_max > kMaxDeg)
    return fail(LIM_E_UNSUPPORTED, "check or qubit degree above LIM_MAX_DEGREE");
  if (out.dc_min < 1) return fail(LIM_E_INVAL, "every check needs at least one qubit");
  if (mz > 0) {
    // H_Z H_X^T = 0: every Z row meets every X check an even number of times.
    std::vector<int32_t> cnt(m, 0), touched;
    for (int r = 0; r < mz; r++) {
      touched.clear();
      for (int j = hz_ptr[r]; j < hz_ptr[r + 1]; j++) {
        int v = hz_col[j];
        for (int t = out.v_ptr[v]; t < out.v_ptr[v + 1]; t++) {
          int c = out.v_chk[t];
          if (cnt[c]++ == 0) touched.push_back(c);
        }
      }
      for (int c : touched) {
        if (cnt[c] & 1) return fail(LIM_E_NOT_CSS, "H_Z H_X^T != 0");
        cnt[c] = 0;
      }
    }
  }
  int nw = (n + 31) / 32;
  if (logicals) {
    if (k < 0 || k > LIM_MAX_LOGICALS) return fail(LIM_E_UNSUPPORTED, "k out of range");
    out.k = k;
    out.logicals.assign(logicals, logicals + (size_t)k * nw);
    uint32_t tail = (n % 32) ? ((1u << (n % 32)) - 1u) : 0xffffffffu;
    for (int j = 0; j < k; j++) out.logicals[(size_t)j * nw + nw - 1] &= tail;
  } else {
    std::vector<int32_t> zp, zc;
    if (mz > 0) {
      zp.assign(hz_ptr, hz_ptr + mz + 1);
      zc.assign(hz_col, hz_col + hz_ptr[mz]);
    }
    st = logicals_from_hz(n, out.c_ptr, out.c_var, zp, zc, out.logicals, out.k);
    if (st) return st;
  }
  return LIM_OK;
}

int build_rep(int32_t d, int periodic, HostCode &out) {
  if (d < 2) return fail(LIM_E_INVAL, "repetition code needs d >= 2");
  int m = periodic ? d : d - 1;
  std::vector<std::vector<int32_t>> rows;
  for (int c = 0; c < m; c++) rows.push_back(gf2_row({c, (c + 1) % d}));
  std::vector<std::vector<int32_t>> lg = {{0}};  // X on qubit 0 detects the all-ones residual
  return assemble(d, rows, nullptr, &lg, out);
}

int build_toric2d(int32_t L, HostCode &out) {
  if (L < 2) return fail(LIM_E_INVAL, "toric code needs L >= 2");
  auto vid = [L](int x, int y) { return ((y % L + L) % L) * L + ((x % L + L) % L); };
  std::vector<std::vector<int32_t>> rows;
  for (int y = 0; y < L; y++)
    for (int x = 0; x < L; x++) {
      int c = vid(x, y);
      rows.push_back(gf2_row({2 * c, 2 * c + 1, 2 * vid(x - 1, y), 2 * vid(x, y - 1) + 1}));
    }
  std::vector<std::vector<int32_t>> lg(2);
  for (int y = 0; y < L; y++) lg[0].push_back(2 * vid(0, y));
  for (int x = 0; x < L; x++) lg[1].push_back(2 * vid(x, 0) + 1);
  return assemble(2 * L * L, rows, nullptr, &lg, out);
}

int build_toric3d(int32_t L, int sector, HostCode &out) {
  if (L < 2) return fail(LIM_E_INVAL, "toric code needs L >= 2");
  if (sector != LIM_SECTOR_POINT && sector != LIM_SECTOR_MEMBRANE)
    return fail(LIM_E_INVAL, "unknown sector");
  auto vid = [L](int x, int y, int z) {
    auto w = [L](int a) { return ((a % L) + L) % L; };
    return (w(z) * L + w(y)) * L + w(x);
  };
  std::vector<std::vector<int32_t>> rows;
  std::vector<std::vector<int32_t>> lg(3);
  if (sector == LIM_SECTOR_POINT) {
    for (int z = 0; z < L; z++)
      for (int y = 0; y < L; y++)
        for (int x = 0; x < L; x++) {
          int v[3] = {x, y, z};
          std::vector<int32_t> r;
          for (int a = 0; a < 3; a++) {
            int vm[3] = {x, y, z};
            vm[a]--;
            r.push_back(3 * vid(v[0], v[1], v[2]) + a);
            r.push_back(3 * vid(vm[0], vm[1], vm[2]) + a);
          }
          rows.push_back(gf2_row(r));
          for (int a = 0; a < 3; a++)
            if (v[a] == 0) lg[a].push_back(3 * vid(x, y, z) + a);
        }
  } else {
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int z = 0; z < L; z++)
      for (int y = 0; y < L; y++)
        for (int x = 0; x < L; x++)
          for (auto &pr : pairs) {
            int a = pr[0], b = pr[1];
            int va[3] = {x, y, z}, vb[3] = {x, y, z};
            va[a]++;
            vb[b]++;
            rows.push_back(gf2_row({3 * vid(x, y, z) + a, 3 * vid(va[0], va[1], va[2]) + b,
                                    3 * vid(vb[0], vb[1], vb[2]) + a, 3 * vid(x, y, z) + b}));
          }
    for (int a = 0; a < 3; a++)
      for (int t = 0; t < L; t++) {
        int v[3] = {0, 0, 0};
        v[a] = t;
        lg[a].push_back(3 * vid(v[0], v[1], v[2]) + a);
      }
  }
  return assemble(3 * L * L * L, rows, nullptr, &lg, out);
}

int build_bb(int32_t l, int32_t m, const int32_t *a_xy, const int32_t *b_xy, HostCode &out) {
  if (l < 1 || m < 1 || l * m < 2) return fail(LIM_E_INVAL, "bivariate-bicycle code needs l*m >= 2");
  static const int32_t gross_a[6] = {3, 0, 0, 1, 0, 2};  // x^3 + y + y^2
  static const int32_t gross_b[6] = {0, 3, 1, 0, 2, 0};  // y^3 + x + x^2
  const int32_t *A = a_xy ? a_xy : gross_a;
  const int32_t *B = b_xy ? b_xy : gross_b;
  int lm = l * m;
  auto idx = [l, m](int i, int j) { return (((i % l) + l) % l) * m + (((j % m) + m) % m); };
  std::vector<std::vector<int32_t>> hx, hz;
  for (int i = 0; i < l; i++)
    for (int j = 0; j < m; j++) {
      std::vector<int32_t> rx, rz;
      for (int t = 0; t < 3; t++) {
        rx.push_back(idx(i + A[2 * t], j + A[2 * t + 1]));
        rx.push_back(lm + idx(i + B[2 * t], j + B[2 * t + 1]));
        rz.push_back(idx(i - B[2 * t], j - B[2 * t + 1]));
        rz.push_back(lm + idx(i - A[2 * t], j - A[2 * t + 1]));
      }
      hx.push_back(gf2_row(rx));
      hz.push_back(gf2_row(rz));
    }
  return assemble(2 * lm, hx, &hz, nullptr, out);
}

}  // namespace lim
