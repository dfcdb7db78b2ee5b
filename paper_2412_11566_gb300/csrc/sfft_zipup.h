// Host construction of the SFFT MPO of one axis from the reduced QFT circuit
// (Sec. 4.1: Hadamard and controlled-phase gates without the SWAP network)
// by zip-up sweeps (Sec. 4.2), then one TT rounding. The MPO is tiny (n cores
// of at most 2^min(b, n-b) x 4 x 2^min(b+1, n-b-1) entries), so it is built in
// plain C++ on the host; no GPU is involved.
//
// Core layout: (r, out, in, r') row-major, out/in bits of qubit b, most
// significant first; the operator is S[k', x] = N^-1/2 exp(2 pi i rev(k') x / N).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace qtt_zipup {

using cd = std::complex<double>;

// Row-major dense complex matrix.
struct Mat {
  int m = 0, n = 0;
  std::vector<cd> a;
  Mat() = default;
  Mat(int rows, int cols) : m(rows), n(cols), a((size_t)rows * cols, cd(0, 0)) {}
  cd& at(int i, int j) { return a[(size_t)i * n + j]; }
  const cd& at(int i, int j) const { return a[(size_t)i * n + j]; }
};

// Thin SVD A = U diag(s) Vh by one-sided (Hestenes) Jacobi on the columns of A
// (of A^H when A is wide). For a column pair (p, q) with g = a_p^H a_q, column
// q is first multiplied by the phase conj(g)/|g| so that the pair's Gram entry
// is real, then a real Jacobi rotation orthogonalises the pair; the same
// unitary goes into V. Sweeps run until every pair is orthogonal to 1e-15
// relative or involves a column below 1e-16 ||A||_F, at most 60. Singular values come out descending; U's column for a
// zero singular value is left zero.
inline void svd(const Mat& A, Mat& U, std::vector<double>& s, Mat& Vh) {
  if (A.m < A.n) {  // A = (A^H)^H = (U' S V'^H)^H
    Mat Ah(A.n, A.m);
    for (int i = 0; i < A.m; ++i)
      for (int j = 0; j < A.n; ++j) Ah.at(j, i) = std::conj(A.at(i, j));
    Mat U2, Vh2;
    svd(Ah, U2, s, Vh2);
    const int k = (int)s.size();
    U = Mat(A.m, k);
    for (int i = 0; i < A.m; ++i)
      for (int j = 0; j < k; ++j) U.at(i, j) = std::conj(Vh2.at(j, i));
    Vh = Mat(k, A.n);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < A.n; ++i) Vh.at(j, i) = std::conj(U2.at(i, j));
    return;
  }
  const int m = A.m, n = A.n;
  Mat W = A, V(n, n);
  for (int j = 0; j < n; ++j) V.at(j, j) = cd(1, 0);
  double frob2 = 0;
  for (const cd& z : A.a) frob2 += std::norm(z);
  // columns below the rounding level of ||A||_F are numerically zero: pairs
  // of them carry no information and would keep the sweeps from settling
  const double negligible = 1e-32 * frob2;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0, beta = 0;
        cd g(0, 0);
        for (int i = 0; i < m; ++i) {
          alpha += std::norm(W.at(i, p));
          beta += std::norm(W.at(i, q));
          g += std::conj(W.at(i, p)) * W.at(i, q);
        }
        const double ag = std::abs(g);
        if (ag == 0.0 || ag <= 1e-15 * std::sqrt(alpha * beta)) continue;
        if (alpha <= negligible || beta <= negligible) continue;
        rotated = true;
        const cd ph = std::conj(g) / ag;  // column q times ph: Gram entry becomes |g|
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int i = 0; i < m; ++i) {
          const cd wp = W.at(i, p), wq = W.at(i, q) * ph;
          W.at(i, p) = c * wp - sn * wq;
          W.at(i, q) = sn * wp + c * wq;
        }
        for (int i = 0; i < n; ++i) {
          const cd vp = V.at(i, p), vq = V.at(i, q) * ph;
          V.at(i, p) = c * vp - sn * vq;
          V.at(i, q) = sn * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int i = 0; i < m; ++i) acc += std::norm(W.at(i, j));
    nrm[j] = std::sqrt(acc);
  }
  std::vector<int> order(n);
  for (int j = 0; j < n; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  s.assign(n, 0.0);
  U = Mat(m, n);
  Vh = Mat(n, n);
  for (int jj = 0; jj < n; ++jj) {
    const int j = order[jj];
    s[jj] = nrm[j];
    if (nrm[j] > 0)
      for (int i = 0; i < m; ++i) U.at(i, jj) = W.at(i, j) / nrm[j];
    for (int i = 0; i < n; ++i) Vh.at(jj, i) = std::conj(V.at(i, j));
  }
}

// An MPO core (r, out = 2, in = 2, r').
struct Core {
  int r0 = 1, r1 = 1;
  std::vector<cd> a;  // r0 * 4 * r1
  Core() = default;
  Core(int a0, int a1) : r0(a0), r1(a1), a((size_t)a0 * 4 * a1, cd(0, 0)) {}
  cd& at(int x, int o, int i, int y) { return a[(((size_t)x * 2 + o) * 2 + i) * r1 + y]; }
  const cd& at(int x, int o, int i, int y) const { return a[(((size_t)x * 2 + o) * 2 + i) * r1 + y]; }
};
using Mpo = std::vector<Core>;

inline Mpo identity_mpo(int n) {
  Mpo op(n, Core(1, 1));
  for (auto& c : op) c.at(0, 0, 0, 0) = c.at(0, 1, 1, 0) = cd(1, 0);
  return op;
}

// Gate MPOs of the reduced QFT circuit, one per qubit, in the order they
// act. For qubit q: H on q followed by cP(pi / 2^(m - q)) between q and every
// less significant qubit m > q. The controlled phases are diagonal and
// commute, so (as Sec. 4.2 recombines the split copy tensors) they merge
// with H into one MPO of bond 2: site q applies H and copies its output bit
// into the bond; each later site passes the bond on and multiplies by
// e^{i pi / 2^(m - q)} when the bond and its own bit are both 1; the last
// site closes the bond. n zip-ups instead of n (n + 1) / 2.
inline std::vector<Mpo> qft_gates(int n) {
  std::vector<Mpo> gates;
  const double h = 1.0 / std::sqrt(2.0);
  const double pi = 3.14159265358979323846;
  const double H[2][2] = {{h, h}, {h, -h}};
  for (int q = 0; q < n; ++q) {
    Mpo g = identity_mpo(n);
    if (q == n - 1) {
      g[q] = Core(1, 1);
      for (int o = 0; o < 2; ++o)
        for (int i = 0; i < 2; ++i) g[q].at(0, o, i, 0) = cd(H[o][i], 0);
      gates.push_back(g);
      continue;
    }
    g[q] = Core(1, 2);
    for (int o = 0; o < 2; ++o)
      for (int i = 0; i < 2; ++i) g[q].at(0, o, i, o) = cd(H[o][i], 0);
    for (int m = q + 1; m < n; ++m) {
      const int rout = m == n - 1 ? 1 : 2;
      Core c(2, rout);
      const cd ph = std::polar(1.0, pi / (double)(1 << (m - q)));
      for (int bnd = 0; bnd < 2; ++bnd)
        for (int o = 0; o < 2; ++o)
          c.at(bnd, o, o, rout == 1 ? 0 : bnd) = (bnd == 1 && o == 1) ? ph : cd(1, 0);
      g[m] = c;
    }
    gates.push_back(g);
  }
  return gates;
}

// G W (W acts first) by a zip-up sweep: left to right, the carried factor is
// contracted with the site's two cores, reshaped to (carried rank x out x in,
// bond of G x bond of W) and split by an SVD that keeps the singular values
// above rel_tol times the largest; S V^H moves on to the next site.
inline Mpo zipup(const Mpo& G, const Mpo& W, double rel_tol) {
  const int n = (int)W.size();
  Mpo out(n);
  int R = 1, cg = 1, cw = 1;
  std::vector<cd> carry(1, cd(1, 0));  // (R, cg, cw)
  for (int b = 0; b < n; ++b) {
    const Core& g = G[b];
    const Core& w = W[b];
    const int h = g.r1, v = w.r1;
    // T[R, o, i, h, v] = sum_{x, y, m} carry[R, x, y] g[x, o, m, h] w[y, m, i, v]
    Mat T(R * 4, h * v);
    for (int rr = 0; rr < R; ++rr)
      for (int x = 0; x < cg; ++x)
        for (int y = 0; y < cw; ++y) {
          const cd cf = carry[((size_t)rr * cg + x) * cw + y];
          if (cf == cd(0, 0)) continue;
          for (int o = 0; o < 2; ++o)
            for (int mm = 0; mm < 2; ++mm)
              for (int hh = 0; hh < h; ++hh) {
                const cd gv = g.at(x, o, mm, hh);
                if (gv == cd(0, 0)) continue;
                for (int i = 0; i < 2; ++i)
                  for (int vv = 0; vv < v; ++vv)
                    T.at((rr * 2 + o) * 2 + i, hh * v + vv) += cf * gv * w.at(y, mm, i, vv);
              }
        }
    if (b == n - 1) {
      out[b] = Core(R, 1);
      for (int row = 0; row < R * 4; ++row) out[b].a[row] = T.at(row, 0);  // h * v == 1
      break;
    }
    Mat U, Vh;
    std::vector<double> s;
    svd(T, U, s, Vh);
    int k = 0;
    while (k < (int)s.size() && s[k] > rel_tol * s[0]) ++k;
    k = std::max(k, 1);
    out[b] = Core(R, k);
    for (int row = 0; row < R * 4; ++row)
      for (int j = 0; j < k; ++j) out[b].a[(size_t)row * k + j] = U.at(row, j);
    carry.assign((size_t)k * h * v, cd(0, 0));
    for (int j = 0; j < k; ++j)
      for (int col = 0; col < h * v; ++col) carry[(size_t)j * h * v + col] = s[j] * Vh.at(j, col);
    R = k;
    cg = h;
    cw = v;
  }
  return out;
}

// TT rounding of an MPO seen as a TT with mode size 4 (Sec. 3): left-to-right
// orthogonalisation (by SVD), then right-to-left truncated SVDs keeping, per
// bond, the smallest rank whose discarded tail sum s^2 is within
// (eps ||op|| / sqrt(n - 1))^2.
inline Mpo round_mpo(Mpo op, double eps) {
  const int n = (int)op.size();
  for (int k = 0; k + 1 < n; ++k) {
    Core& c = op[k];
    Mat M(c.r0 * 4, c.r1);
    M.a = c.a;
    Mat U, Vh;
    std::vector<double> s;
    svd(M, U, s, Vh);
    const int kk = (int)s.size();
    Core nc(c.r0, kk);
    for (int row = 0; row < c.r0 * 4; ++row)
      for (int j = 0; j < kk; ++j) nc.a[(size_t)row * kk + j] = U.at(row, j);
    // next core <- (S Vh) next
    Core& d = op[k + 1];
    Core nd(kk, d.r1);
    for (int j = 0; j < kk; ++j)
      for (int y = 0; y < c.r1; ++y) {
        const cd f = s[j] * Vh.at(j, y);
        if (f == cd(0, 0)) continue;
        for (int e = 0; e < 4 * d.r1; ++e) nd.a[(size_t)j * 4 * d.r1 + e] += f * d.a[(size_t)y * 4 * d.r1 + e];
      }
    op[k] = nc;
    op[k + 1] = nd;
  }
  double nrm2 = 0;
  for (const cd& z : op[n - 1].a) nrm2 += std::norm(z);
  const double delta2 = eps * eps * nrm2 / std::max(n - 1, 1);
  for (int k = n - 1; k >= 1; --k) {
    Core& c = op[k];
    Mat M(c.r0, 4 * c.r1);
    M.a = c.a;
    Mat U, Vh;
    std::vector<double> s;
    svd(M, U, s, Vh);
    int kk = (int)s.size();
    double tail = 0;
    while (kk > 1 && tail + s[kk - 1] * s[kk - 1] <= delta2) {
      tail += s[kk - 1] * s[kk - 1];
      --kk;
    }
    Core nc(kk, c.r1);
    for (int j = 0; j < kk; ++j)
      for (int e = 0; e < 4 * c.r1; ++e) nc.a[(size_t)j * 4 * c.r1 + e] = Vh.at(j, e);
    // previous core <- previous (U S)
    Core& p = op[k - 1];
    Core np(p.r0, kk);
    for (int row = 0; row < p.r0 * 4; ++row)
      for (int y = 0; y < c.r0; ++y) {
        const cd f = p.a[(size_t)row * c.r0 + y];
        if (f == cd(0, 0)) continue;
        for (int j = 0; j < kk; ++j) np.a[(size_t)row * kk + j] += f * U.at(y, j) * s[j];
      }
    op[k] = nc;
    op[k - 1] = np;
  }
  return op;
}

// The circuit is G_{n-1} ... G_1 G_0 (G_0 acts first); the product is
// formed from the other end, P <- P G_q for q = n - 1 down to 0, so that each
// partial product is the reduced QFT of the last n - q qubits. A zip-up sweep
// alone cannot truncate well (the part to the right of the split is not
// orthonormal, so its local singular values are not the bond's): its ranks
// double with every gate, up to 2^(n-1) (512 at n = 10). Each partial product
// is therefore rounded at eps / 100, which keeps its ranks at their true
// values (about a dozen), and the result is rounded once more at eps.
inline Mpo sfft_mpo(int n, double eps) {
  const std::vector<Mpo> gates = qft_gates(n);
  Mpo op = identity_mpo(n);
  for (int q = n - 1; q >= 0; --q) op = round_mpo(zipup(op, gates[q], 1e-2 * eps), 1e-2 * eps);
  return round_mpo(op, eps);
}

}  // namespace qtt_zipup
