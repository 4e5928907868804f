// Host-side FP64 setup numerics (no CUDA): GLL basis, 1D operators, the
// symmetric eigen-solver and the per-level tables.
#pragma once

#include <vector>

namespace semmg {

// Largest number of inverse-eigenvalue entries precomputed per level (element
// and element-centred block classes; the star classes of an FP64 V-cycle may
// take up to kMaxStarRtabFp64 entries, built on the device).
constexpr size_t kMaxRtabEntries = size_t(1) << 25;
constexpr size_t kMaxStarRtabFp64 = size_t(1) << 29;

struct HostLevel {
  int p = 0;
  double lam = 0.0;
  std::vector<double> x, w, Ls;                    // GLL nodes, weights, standard stiffness
  std::vector<double> Sref, Sh, a0, ap, lamI;      // interior eigen-tables (columns: even, then odd eigenvectors)
  std::vector<double> hval[3];                     // distinct element widths per axis
  std::vector<int> hcls[3];                        // width class of every element per axis
  std::vector<double> Relem;                       // per width-class triple [k3][k2][k1]: 1/(lam + sum 4/h^2 Lam)
  std::vector<double> starS[3], starLam[3];        // per axis: (n_d+1) blocks
  std::vector<unsigned char> act[3];
  std::vector<unsigned char> sym[3];               // per vertex line: centrosymmetric (folded) tables
  std::vector<int> cls[3], rep[3];                 // line class per vertex line, representative line per class
  std::vector<double> w1d;                         // smoother weights at |offset|
  std::vector<double> J;                           // interpolation from the next coarser level
  int pc = 0;
  // element-centred blocks (Sec. 3.4), built on request: per axis n_d block lines of
  // nE x nE eigenvectors (and their transposes), nE eigenvalues and nE weight factors
  // (nE = 3p - 1); lines with equal tables share a class, and per class triple
  // 1/(lam + Lam1 + Lam2 + Lam3) is tabulated when small enough
  std::vector<double> ebS[3], ebST[3], ebLam[3], ebW[3];
  std::vector<int> ebCls[3], ebRep[3];
  std::vector<double> ebR;
};

struct HostCoarse {
  int K[3] = {0, 0, 0};
  int g0[3] = {1, 1, 1};
  std::vector<double> S[3], lam[3];
};

void gll_host(int p, std::vector<double>& x, std::vector<double>& w);
void deriv_matrix(int p, const std::vector<double>& x, std::vector<double>& D);
void stiffness(int p, const std::vector<double>& x, const std::vector<double>& w, std::vector<double>& L);
void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& xf, std::vector<double>& J);
void jacobi_eig(int n, std::vector<double> A, std::vector<double>& ev, std::vector<double>& V);
void gen_eig_diag_mass(int n, const std::vector<double>& L, const std::vector<double>& Md, std::vector<double>& S,
                       std::vector<double>& lam);
void gen_eig_centrosym(int n, const std::vector<double>& L, const std::vector<double>& Md, std::vector<double>& S,
                       std::vector<double>& lam);
double weight_poly(double t);
// bc: faces -x1, +x1, -x2, +x2, -x3, +x3, SEMMG_BC_DIRICHLET or SEMMG_BC_NEUMANN
void build_level_tables(HostLevel& L, const std::vector<double>* h, const int* bc);
void build_coarse_tables(int p0, const std::vector<double>* h, const int* bc, HostCoarse& C);
// element-centred block tables of a level whose GLL tables are built (needs 3 elements per periodic axis);
// weights: SEMMG_SMOOTHER_ELEMENT or SEMMG_SMOOTHER_ELEMENT_MULT
void build_eblock_tables(HostLevel& L, const std::vector<double>* h, const int* bc, int weights);

}  // namespace semmg
