// Host-side FP64 setup numerics: GLL basis, 1D operators, symmetric eigen-
// solver, and the per-level tables of Sec. 2-4.  Runs once per semmg_setup.
#include "setup_host.h"

#include "semmg.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace semmg {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *P = p1;
  // P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); only used for |x| < 1
  *dP = (std::fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.0;
}

void gll_host(int p, std::vector<double>& x, std::vector<double>& w) {
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  // interior nodes: roots of P_p', Newton from the Chebyshev-Lobatto points;
  // with q = P_p', q' = (2 x P_p' - p (p+1) P_p) / (1 - x^2) (Legendre ODE)
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, &P, &dP);
      const double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      const double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  std::sort(x.begin(), x.end());
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  // the rule is symmetric about 0; make it exactly so (x_i = -x_{p-i}, w_i = w_{p-i})
  for (int i = 0; i <= p / 2; ++i) {
    const double xs = 0.5 * (x[p - i] - x[i]), ws = 0.5 * (w[i] + w[p - i]);
    x[i] = -xs;
    x[p - i] = xs;
    w[i] = w[p - i] = ws;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
}

// D[i][j] = l_j'(x_i) through the Legendre form of the GLL cardinal functions.
void deriv_matrix(int p, const std::vector<double>& x, std::vector<double>& D) {
  D.assign((p + 1) * (p + 1), 0.0);
  std::vector<double> P(p + 1);
  for (int i = 0; i <= p; ++i) {
    double dP;
    legendre(p, x[i], &P[i], &dP);
  }
  for (int i = 0; i <= p; ++i)
    for (int j = 0; j <= p; ++j) {
      if (i != j)
        D[i * (p + 1) + j] = P[i] / (P[j] * (x[i] - x[j]));
      else if (i == 0)
        D[0] = -0.25 * p * (p + 1.0);
      else if (i == p)
        D[p * (p + 1) + p] = 0.25 * p * (p + 1.0);
    }
}

void stiffness(int p, const std::vector<double>& x, const std::vector<double>& w, std::vector<double>& L) {
  std::vector<double> D;
  deriv_matrix(p, x, D);
  const int P1 = p + 1;
  L.assign(P1 * P1, 0.0);
  for (int i = 0; i < P1; ++i)
    for (int j = 0; j < P1; ++j) {
      double s = 0.0;
      for (int q = 0; q < P1; ++q) s += w[q] * D[q * P1 + i] * D[q * P1 + j];
      L[i * P1 + j] = s;
    }
  for (int i = 0; i < P1; ++i)
    for (int j = i + 1; j < P1; ++j) {
      const double a = 0.5 * (L[i * P1 + j] + L[j * P1 + i]);
      L[i * P1 + j] = L[j * P1 + i] = a;
    }
  // centrosymmetric: L[i][j] = L[p-i][p-j]
  for (int i = 0; i < P1; ++i)
    for (int j = 0; j < P1; ++j) {
      const int i2 = p - i, j2 = p - j;
      if (i * P1 + j < i2 * P1 + j2) {
        const double a = 0.5 * (L[i * P1 + j] + L[i2 * P1 + j2]);
        L[i * P1 + j] = L[i2 * P1 + j2] = a;
      }
    }
}

// J[I][i] = prod_{k != i} (xf_I - xc_k) / (xc_i - xc_k)
void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& xf, std::vector<double>& J) {
  const int nc = (int)xc.size(), nf = (int)xf.size();
  J.assign(nf * nc, 0.0);
  for (int I = 0; I < nf; ++I)
    for (int i = 0; i < nc; ++i) {
      double v = 1.0;
      for (int k = 0; k < nc; ++k)
        if (k != i) v *= (xf[I] - xc[k]) / (xc[i] - xc[k]);
      J[I * nc + i] = v;
    }
}

// Cyclic Jacobi rotations for a symmetric matrix A (n x n, row-major):
// A = V diag(ev) V^T, V orthogonal (columns are eigenvectors).
void jacobi_eig(int n, std::vector<double> A, std::vector<double>& ev, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double scale = 0.0;
  for (double a : A) scale = std::max(scale, std::fabs(a));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off == 0.0 || off <= 1e-36 * scale * scale) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) <= 1e-19 * (std::fabs(A[p * n + p]) + std::fabs(A[q * n + q]))) {
          A[p * n + q] = A[q * n + p] = 0.0;
          continue;
        }
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
}

// Generalised problem L S = M S Lam with diagonal M > 0: S^T M S = I, S^T L S = Lam.
void gen_eig_diag_mass(int n, const std::vector<double>& L, const std::vector<double>& Md, std::vector<double>& S,
                       std::vector<double>& lam) {
  std::vector<double> A(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = L[i * n + j] / std::sqrt(Md[i] * Md[j]);
  std::vector<double> Q;
  jacobi_eig(n, A, lam, Q);
  S.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) S[i * n + k] = Q[i * n + k] / std::sqrt(Md[i]);
}

// Centrosymmetric generalised problem (L, diag M) on n points (L[i][j] =
// L[n-1-i][n-1-j], M likewise): eigenvectors split into even (v[i] =
// v[n-1-i]) and odd (v[i] = -v[n-1-i]) ones, computed separately in the
// folded bases.  With h = n/2 (rounded down) and ne = (n+1)/2, the columns of
// S hold the ne even eigenvectors first, then the n - ne odd ones.  The
// folded coordinates are: even position j < ne pairs rows h+j and n-1-(h+j)
// (the centre alone when they coincide); odd position q >= ne pairs rows q
// and n-1-q.
void gen_eig_centrosym(int n, const std::vector<double>& L, const std::vector<double>& Md, std::vector<double>& S,
                       std::vector<double>& lam) {
  const int h = n / 2, ne = (n + 1) / 2, no = n - ne;
  std::vector<double> A(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = L[i * n + j] / std::sqrt(Md[i] * Md[j]);
  const double r2 = 1.0 / std::sqrt(2.0);
  std::vector<std::vector<double>> E(ne, std::vector<double>(n, 0.0)), O(no, std::vector<double>(n, 0.0));
  for (int j = 0; j < ne; ++j) {
    const int i = h + j, mi = n - 1 - i;
    if (i == mi) E[j][i] = 1.0;
    else { E[j][i] = r2; E[j][mi] = r2; }
  }
  for (int q = ne; q < n; ++q) {
    O[q - ne][q] = r2;
    O[q - ne][n - 1 - q] = -r2;
  }
  auto project = [&](const std::vector<std::vector<double>>& B, std::vector<double>& P) {
    const int k = (int)B.size();
    P.assign(k * k, 0.0);
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) {
          if (B[a][i] == 0.0) continue;
          for (int j = 0; j < n; ++j) sum += B[a][i] * A[i * n + j] * B[b][j];
        }
        P[a * k + b] = sum;
      }
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b) P[a * k + b] = P[b * k + a] = 0.5 * (P[a * k + b] + P[b * k + a]);
  };
  std::vector<double> Ae, Ao, Qe, Qo, le, lo;
  project(E, Ae);
  project(O, Ao);
  jacobi_eig(ne, Ae, le, Qe);
  if (no > 0) jacobi_eig(no, Ao, lo, Qo);
  S.assign(n * n, 0.0);
  lam.assign(n, 0.0);
  for (int k = 0; k < ne; ++k) {
    lam[k] = le[k];
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < n; ++i) S[i * n + k] += E[a][i] * Qe[a * ne + k];
  }
  for (int k = 0; k < no; ++k) {
    lam[ne + k] = lo[k];
    for (int a = 0; a < no; ++a)
      for (int i = 0; i < n; ++i) S[i * n + (ne + k)] += O[a][i] * Qo[a * no + k];
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) S[i * n + k] /= std::sqrt(Md[i]);
  // exact parity: odd vectors vanish at a centre node, mirrored rows are equal up to sign
  for (int i = 0; i < n; ++i) {
    const int mi = n - 1 - i;
    if (mi < i) continue;
    for (int k = 0; k < n; ++k) {
      if (mi == i) {
        if (k >= ne) S[i * n + k] = 0.0;
      } else {
        const double v = S[mi * n + k];
        S[i * n + k] = k < ne ? v : -v;
      }
    }
  }
}

double weight_poly(double t) {
  const double t2 = t * t, t4 = t2 * t2;
  return 1.0 - 35.0 * t4 + 84.0 * t4 * t - 70.0 * t4 * t2 + 20.0 * t4 * t2 * t;
}

void build_level_tables(HostLevel& L, const std::vector<double>* h, const int* bc) {
  const int p = L.p, m = p - 1, P1 = p + 1, nS = 2 * m + 1;
  gll_host(p, L.x, L.w);
  stiffness(p, L.x, L.w, L.Ls);
  // interior reference eigenpairs (Sec. 3.2 applied to one element's interior)
  L.Sref.clear();
  L.Sh.clear();
  L.a0.clear();
  L.ap.clear();
  L.lamI.clear();
  if (m > 0) {
    std::vector<double> Lii(m * m), Mii(m);
    for (int i = 0; i < m; ++i) {
      Mii[i] = L.w[i + 1];
      for (int j = 0; j < m; ++j) Lii[i * m + j] = L.Ls[(i + 1) * P1 + (j + 1)];
    }
    gen_eig_centrosym(m, Lii, Mii, L.Sref, L.lamI);
    L.Sh.resize(m * m);
    L.a0.assign(m, 0.0);
    L.ap.assign(m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) {
        L.Sh[i * m + k] = L.w[i + 1] * L.Sref[i * m + k];
        L.a0[k] += L.Sref[i * m + k] * L.Ls[(i + 1) * P1 + 0];
        L.ap[k] += L.Sref[i * m + k] * L.Ls[(i + 1) * P1 + p];
      }
  }
  // star tables per axis and vertex line (Sec. 3.2, 3.3)
  for (int d = 0; d < 3; ++d) {
    const int nd = (int)h[d].size();
    const int Nd = nd * p + 1;
    L.starS[d].assign((size_t)(nd + 1) * nS * nS, 0.0);
    L.starLam[d].assign((size_t)(nd + 1) * nS, 1.0);
    L.act[d].assign((size_t)(nd + 1) * nS, 0);
    L.sym[d].assign(nd + 1, 0);
    const bool per = bc[2 * d] == SEMMG_BC_PERIODIC;
    for (int c = 0; c <= nd; ++c) {
      std::vector<double> Mb(nS, 0.0), Lb(nS * nS, 0.0);
      for (int a = c - 1; a <= c; ++a) {
        // on a periodic axis the element beyond an end is the one at the other end
        const int aw = per ? (a + nd) % nd : a;
        if (aw < 0 || aw >= nd) continue;
        const double ha = h[d][aw];
        for (int i = 0; i <= p; ++i) {
          const int ji = a * p + i - c * p;
          if (ji < -m || ji > m) continue;
          Mb[ji + m] += 0.5 * ha * L.w[i];
          for (int k = 0; k <= p; ++k) {
            const int jk = a * p + k - c * p;
            if (jk < -m || jk > m) continue;
            Lb[(ji + m) * nS + (jk + m)] += 2.0 / ha * L.Ls[i * P1 + k];
          }
        }
      }
      // active: nodes that are unknowns of the domain (inside it, not on a Dirichlet face)
      const int glo = bc[2 * d] == SEMMG_BC_DIRICHLET ? 1 : 0;
      const int ghi = bc[2 * d + 1] == SEMMG_BC_DIRICHLET ? Nd - 2 : Nd - 1;
      std::vector<int> act;
      for (int j = -m; j <= m; ++j) {
        const int g = c * p + j;
        if (per || (g >= glo && g <= ghi)) act.push_back(j + m);
      }
      double* S = &L.starS[d][(size_t)c * nS * nS];
      double* lam = &L.starLam[d][(size_t)c * nS];
      unsigned char* ac = &L.act[d][(size_t)c * nS];
      for (int i = 0; i < nS; ++i) S[i * nS + i] = 1.0;  // identity padding
      const int na = (int)act.size();
      const bool sym = per ? (na == nS && h[d][(c + nd - 1) % nd] == h[d][c % nd])
                           : (c >= 1 && c <= nd - 1 && na == nS && h[d][c - 1] == h[d][c]);
      L.sym[d][c] = sym ? 1 : 0;
      if (sym) {
        std::vector<double> Ss, ls;
        gen_eig_centrosym(nS, Lb, Mb, Ss, ls);
        for (int i = 0; i < nS; ++i) {
          ac[i] = 1;
          lam[i] = ls[i];
          for (int k = 0; k < nS; ++k) S[i * nS + k] = Ss[i * nS + k];
        }
      } else if (na > 0) {
        std::vector<double> La(na * na), Ma(na), Sa, la;
        for (int i = 0; i < na; ++i) {
          Ma[i] = Mb[act[i]];
          for (int j = 0; j < na; ++j) La[i * na + j] = Lb[act[i] * nS + act[j]];
        }
        gen_eig_diag_mass(na, La, Ma, Sa, la);
        for (int i = 0; i < na; ++i) {
          S[act[i] * nS + act[i]] = 0.0;
          ac[act[i]] = 1;
          lam[act[i]] = la[i];
        }
        for (int i = 0; i < na; ++i)
          for (int k = 0; k < na; ++k) S[act[i] * nS + act[k]] = Sa[i * na + k];
      }
    }
  }
  // vertex lines with identical tables share a class (uniform meshes: the two
  // boundary lines and one interior class per axis)
  for (int d = 0; d < 3; ++d) {
    const int nl = (int)h[d].size() + 1;
    L.cls[d].assign(nl, -1);
    L.rep[d].clear();
    for (int c = 0; c < nl; ++c) {
      for (int r = 0; r < (int)L.rep[d].size() && L.cls[d][c] < 0; ++r) {
        const int c2 = L.rep[d][r];
        bool same = L.sym[d][c] == L.sym[d][c2];
        for (int i = 0; same && i < nS * nS; ++i)
          same = L.starS[d][(size_t)c * nS * nS + i] == L.starS[d][(size_t)c2 * nS * nS + i];
        for (int i = 0; same && i < nS; ++i)
          same = L.starLam[d][(size_t)c * nS + i] == L.starLam[d][(size_t)c2 * nS + i] &&
                 L.act[d][(size_t)c * nS + i] == L.act[d][(size_t)c2 * nS + i];
        if (same) L.cls[d][c] = r;
      }
      if (L.cls[d][c] < 0) {
        L.cls[d][c] = (int)L.rep[d].size();
        L.rep[d].push_back(c);
      }
    }
  }
  // the inverse 3D eigenvalues 1/(lam + Lam1 + Lam2 + Lam3) per star class are
  // tabulated on the device at upload (the tables of stretched meshes reach GB)
  // element classes: elements with equal widths share their interior eigen-tables,
  // so 1/(lam + sum_d 4/h_d^2 Lam[k_d]) is tabulated per distinct width triple
  for (int d = 0; d < 3; ++d) {
    L.hval[d].clear();
    L.hcls[d].assign(h[d].size(), 0);
    for (size_t a = 0; a < h[d].size(); ++a) {
      int found = -1;
      for (size_t r = 0; r < L.hval[d].size(); ++r)
        if (L.hval[d][r] == h[d][a]) found = (int)r;
      if (found < 0) {
        found = (int)L.hval[d].size();
        L.hval[d].push_back(h[d][a]);
      }
      L.hcls[d][a] = found;
    }
  }
  L.Relem.clear();
  if (m > 0) {
    const size_t n3 = (size_t)m * m * m;
    const size_t ncls = L.hval[0].size() * L.hval[1].size() * L.hval[2].size();
    if (ncls * n3 <= kMaxRtabEntries) {
      L.Relem.resize(ncls * n3);
      size_t o = 0;
      for (double h1 : L.hval[0])
        for (double h2 : L.hval[1])
          for (double h3 : L.hval[2]) {
            const double e1 = 4.0 / (h1 * h1), e2 = 4.0 / (h2 * h2), e3 = 4.0 / (h3 * h3);
            for (int k3 = 0; k3 < m; ++k3)
              for (int k2 = 0; k2 < m; ++k2)
                for (int k1 = 0; k1 < m; ++k1)
                  L.Relem[o++] = 1.0 / (L.lam + e1 * L.lamI[k1] + e2 * L.lamI[k2] + e3 * L.lamI[k3]);
          }
    }
  }
  // smoother weights at star offset |j| (Sec. 3.2): t = (1 + xi_|j|) / 2
  L.w1d.assign(m + 1, 0.0);
  for (int k = 0; k <= m; ++k) L.w1d[k] = weight_poly(0.5 * (1.0 + L.x[k]));
}

// Element-centred blocks (Sec. 3.4): the block of element c spans elements c-1, c, c+1 along
// each axis; its line holds the nE = 3p - 1 nodes strictly inside, j = 0..nE-1 at global
// index (c-1) p + 1 + j.  Assembled 1D matrices of the three elements, identity / 1 padding
// where a node is not an unknown of the domain (ghost element, Dirichlet face, Sec. 3.3).
// Lines with equal inputs (uniform meshes) share one eigen-decomposition.
void build_eblock_tables(HostLevel& L, const std::vector<double>* h, const int* bc, int weights) {
  const int p = L.p, P1 = p + 1, nE = 3 * p - 1;
  for (int d = 0; d < 3; ++d) {
    const int nd = (int)h[d].size();
    const int Nd = nd * p + 1;
    const bool per = bc[2 * d] == SEMMG_BC_PERIODIC;
    const int glo = bc[2 * d] == SEMMG_BC_DIRICHLET ? 1 : 0;
    const int ghi = bc[2 * d + 1] == SEMMG_BC_DIRICHLET ? Nd - 2 : Nd - 1;
    L.ebS[d].assign((size_t)nd * nE * nE, 0.0);
    L.ebLam[d].assign((size_t)nd * nE, 1.0);
    std::vector<std::vector<double>> seenL, seenM;
    std::vector<int>& seenC = L.ebRep[d];
    seenC.clear();
    L.ebCls[d].assign(nd, 0);
    for (int c = 0; c < nd; ++c) {
      std::vector<double> Mb(nE, 0.0), Lb((size_t)nE * nE, 0.0);
      for (int a = c - 1; a <= c + 1; ++a) {
        const int aw = per ? (a + nd) % nd : a;
        if (aw < 0 || aw >= nd) continue;
        const double ha = h[d][aw];
        for (int i = 0; i <= p; ++i) {
          const int ji = (a - c + 1) * p + i - 1;  // block line index of local node i of element a
          if (ji < 0 || ji >= nE) continue;
          Mb[ji] += 0.5 * ha * L.w[i];
          for (int k = 0; k <= p; ++k) {
            const int jk = (a - c + 1) * p + k - 1;
            if (jk < 0 || jk >= nE) continue;
            Lb[(size_t)ji * nE + jk] += 2.0 / ha * L.Ls[i * P1 + k];
          }
        }
      }
      std::vector<int> act;
      for (int j = 0; j < nE; ++j) {
        const int g = (c - 1) * p + 1 + j;
        if (per || (g >= glo && g <= ghi)) act.push_back(j);
      }
      // inactive nodes carry no coupling: zero their rows so equal lines compare equal
      std::vector<char> on(nE, 0);
      for (int j : act) on[j] = 1;
      for (int i = 0; i < nE; ++i)
        if (!on[i]) {
          Mb[i] = 0.0;
          for (int k = 0; k < nE; ++k) Lb[(size_t)i * nE + k] = Lb[(size_t)k * nE + i] = 0.0;
        }
      double* S = &L.ebS[d][(size_t)c * nE * nE];
      double* lam = &L.ebLam[d][(size_t)c * nE];
      int same = -1;
      for (size_t r = 0; r < seenC.size() && same < 0; ++r)
        if (seenL[r] == Lb && seenM[r] == Mb) {
          same = seenC[r];
          L.ebCls[d][c] = (int)r;
        }
      if (same >= 0) {
        std::copy(&L.ebS[d][(size_t)same * nE * nE], &L.ebS[d][(size_t)(same + 1) * nE * nE], S);
        std::copy(&L.ebLam[d][(size_t)same * nE], &L.ebLam[d][(size_t)(same + 1) * nE], lam);
        continue;
      }
      L.ebCls[d][c] = (int)seenC.size();
      seenL.push_back(Lb);
      seenM.push_back(Mb);
      seenC.push_back(c);
      for (int i = 0; i < nE; ++i) S[(size_t)i * nE + i] = 1.0;  // identity padding
      const int na = (int)act.size();
      if (na == 0) continue;
      std::vector<double> La((size_t)na * na), Ma(na), Sa, la;
      for (int i = 0; i < na; ++i) {
        Ma[i] = Mb[act[i]];
        for (int j = 0; j < na; ++j) La[(size_t)i * na + j] = Lb[(size_t)act[i] * nE + act[j]];
      }
      gen_eig_diag_mass(na, La, Ma, Sa, la);
      for (int i = 0; i < na; ++i) {
        S[(size_t)act[i] * nE + act[i]] = 0.0;
        lam[act[i]] = la[i];
      }
      for (int i = 0; i < na; ++i)
        for (int k = 0; k < na; ++k) S[(size_t)act[i] * nE + act[k]] = Sa[(size_t)i * na + k];
    }
    // 1D weight factor of block line c at index j (global node (c-1) p + 1 + j):
    // SEMMG_SMOOTHER_ELEMENT: 1 strictly inside element c, 1/2 on its two faces when the
    // neighbour block beyond exists (else 1), 0 elsewhere;
    // SEMMG_SMOOTHER_ELEMENT_MULT: 1 / (number of blocks c' with (c'-1) p < g < (c'+2) p)
    L.ebW[d].assign((size_t)nd * nE, 0.0);
    for (int c = 0; c < nd; ++c)
      for (int j = 0; j < nE; ++j) {
        double w = 0.0;
        if (weights == SEMMG_SMOOTHER_ELEMENT) {
          const int o = j + 1;  // offset from the block's low end, p and 2p on the element's faces
          if (o > p && o < 2 * p) w = 1.0;
          if (o == p) w = (c > 0 || per) ? 0.5 : 1.0;
          if (o == 2 * p) w = (c < nd - 1 || per) ? 0.5 : 1.0;
        } else {
          int g = (c - 1) * p + 1 + j;
          if (per) g = ((g % (nd * p)) + nd * p) % (nd * p);
          int cnt = 0;
          for (int c2 = 0; c2 < nd; ++c2) {
            int o = g - (c2 - 1) * p;
            if (per) o = ((o % (nd * p)) + nd * p) % (nd * p);
            if (o >= 1 && o <= 3 * p - 1) ++cnt;
          }
          w = cnt > 0 ? 1.0 / cnt : 0.0;
        }
        L.ebW[d][(size_t)c * nE + j] = w;
      }
    L.ebST[d].resize(L.ebS[d].size());
    for (int c = 0; c < nd; ++c)
      for (int j = 0; j < nE; ++j)
        for (int k = 0; k < nE; ++k)
          L.ebST[d][((size_t)c * nE + k) * nE + j] = L.ebS[d][((size_t)c * nE + j) * nE + k];
  }
  // 1/(lam + Lam1[k1] + Lam2[k2] + Lam3[k3]) per class triple, index ((cl3 ncls2 + cl2) ncls1 + cl1)
  const size_t n3 = (size_t)nE * nE * nE;
  const size_t ncls = L.ebRep[0].size() * L.ebRep[1].size() * L.ebRep[2].size();
  L.ebR.clear();
  if (ncls * n3 <= kMaxRtabEntries) {
    L.ebR.resize(ncls * n3);
    size_t o = 0;
    for (int r3 : L.ebRep[2])
      for (int r2 : L.ebRep[1])
        for (int r1 : L.ebRep[0]) {
          const double* l1 = &L.ebLam[0][(size_t)r1 * nE];
          const double* l2 = &L.ebLam[1][(size_t)r2 * nE];
          const double* l3 = &L.ebLam[2][(size_t)r3 * nE];
          for (int k3 = 0; k3 < nE; ++k3)
            for (int k2 = 0; k2 < nE; ++k2)
              for (int k1 = 0; k1 < nE; ++k1) L.ebR[o++] = 1.0 / (L.lam + l1[k1] + l2[k2] + l3[k3]);
        }
  }
}

void build_coarse_tables(int p0, const std::vector<double>* h, const int* bc, HostCoarse& C) {
  std::vector<double> x, w, Ls;
  gll_host(p0, x, w);
  stiffness(p0, x, w, Ls);
  const int P1 = p0 + 1;
  for (int d = 0; d < 3; ++d) {
    const int nd = (int)h[d].size();
    const bool per = bc[2 * d] == SEMMG_BC_PERIODIC;
    const int N = per ? nd * p0 : nd * p0 + 1;  // periodic: the last plane is the first
    const int glo = bc[2 * d] == SEMMG_BC_DIRICHLET ? 1 : 0;
    const int ghi = bc[2 * d + 1] == SEMMG_BC_DIRICHLET ? N - 2 : N - 1;
    const int K = ghi - glo + 1;
    C.g0[d] = glo;
    C.K[d] = K > 0 ? K : 0;
    C.S[d].clear();
    C.lam[d].clear();
    if (K <= 0) continue;
    std::vector<double> Mg(N, 0.0), Lg((size_t)N * N, 0.0);
    for (int a = 0; a < nd; ++a)
      for (int i = 0; i <= p0; ++i) {
        const int gi = (a * p0 + i) % N;
        Mg[gi] += 0.5 * h[d][a] * w[i];
        for (int k = 0; k <= p0; ++k) Lg[(size_t)gi * N + (a * p0 + k) % N] += 2.0 / h[d][a] * Ls[i * P1 + k];
      }
    std::vector<double> Li((size_t)K * K), Mi(K);
    for (int i = 0; i < K; ++i) {
      Mi[i] = Mg[i + glo];
      for (int j = 0; j < K; ++j) Li[(size_t)i * K + j] = Lg[(size_t)(i + glo) * N + (j + glo)];
    }
    gen_eig_diag_mass(K, Li, Mi, C.S[d], C.lam[d]);
  }
}

}  // namespace semmg
