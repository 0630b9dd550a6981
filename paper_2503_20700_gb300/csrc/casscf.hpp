// CAS-SCF device routines (orbital rotation, integral transform, active space,
// orbital gradient).  Host arrays in and out; all arithmetic on the device.
#pragma once
#include "backend.hpp"

namespace dmrg {

class Casscf {
 public:
  struct Dev;
  explicit Casscf(Backend* be);
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
  // device scaling-and-squaring exponential: dR = expm(sign * dK)
  void expm_neg(const double* dK, int n, double* dR, double sign);

 private:
  Backend* be_;
};

}  // namespace dmrg
