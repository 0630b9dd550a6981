// CAS-SCF device routines (orbital rotation, integral transform, active space,
// orbital gradient).  Host arrays in and out; all arithmetic on the device.
#pragma once
#include <vector>

#include "backend.hpp"

namespace dmrg {

class Casscf {
 public:
  struct Dev;
  explicit Casscf(Backend* be);
  // C = A B (n x n, host arrays)
  void matmul(const double* A, const double* B, int n, double* C);
  // R = expm(-K) (U = exp(-kappa) of Sec. II.A)
  void rotation(const double* K, int nb, double* R);
  // dE/dkappa (antisymmetric) for R = expm(-K) given G = dE/dR
  void rotation_backward(const double* K, const double* G, int nb, double* dK);
  // h' = R^T h R, L'^k = R^T L^k R
  void transform(const double* R, const double* h, const double* L, int rank, int nb, double* h_out,
                 double* L_out);
  // closed-shell core energy, inactive-Fock active block and (tu|vw)
  void active_space(const double* h, const double* L, int rank, int nb, int ncore, int ncas,
                    double* e_core, double* h_act, double* eri_act);
  // grad = 2 (F - F^T) (active-active zero); fock (optional) = F
  void gradient(const double* h, const double* L, int rank, int nb, int ncore, int ncas,
                const double* gamma, const double* Gamma, double* grad, double* fock);
  // backward of the whole forward map (rotation, transform, active space)
  // for upstream weights (g_core, g_h, g_eri): the gradient with respect to
  // the full antisymmetric K (nb x nb)
  void transform_backward(const double* K, const double* R, const double* h, const double* L, int rank,
                          int nb, int ncore, int ncas, double g_core, const double* g_h,
                          const double* g_eri, double* dK);
  // device scaling-and-squaring exponential: dR = expm(sign * dK)
  void expm_neg(const double* dK, int n, double* dR, double sign);

 private:
  // device-pointer forms
  void rotation_backward_dev(const double* dK, const double* dG, int nb, double scale, double* ddK);

 public:
  // generalised Fock matrix F of device integrals and RDMs (device), and
  // optionally the diagonal of F^I + F^A (fdiag, nb)
  void fock_dev(const double* dh, const double* dL, int rank, int nb, int ncore, int ncas, const double* dg,
                const double* dG, double* F, double* fdiag = nullptr);

 private:
  Backend* be_;
};

// One DMRG-SCF orbital step per macro iteration (Sec. II.A): limited-memory
// BFGS over the non-redundant rotations with the approximate diagonal
// Hessian as the initial inverse, largest entry capped; history on the
// device.
class ScfStepper {
 public:
  ScfStepper(Backend* be, int nb, int ncore, int ncas, int memory, double max_step);
  ~ScfStepper();
  // masks the gradient matrix (host, nb x nb) to the non-redundant rotations
  // and returns its largest magnitude
  double gradient_max(const double* g_host);
  // the step from the gradient of the last gradient_max call: K (host, nb x nb,
  // antisymmetric) with U <- U expm(-K)
  void step(Casscf& cas, const double* h, const double* L, int rank, const double* gamma, const double* Gamma,
            double* K_host);

 private:
  double dot(const double* a, const double* b);
  Backend* be_;
  int nb_, ncore_, ncas_, memory_;
  double max_step_;
  std::vector<double*> mem_, S_, Y_;
  double *mask_, *g_, *gprev_, *xprev_, *q_, *r_, *hd_, *scal_;
  int pairs_ = 0;
  bool have_prev_ = false;
};

}  // namespace dmrg
