// CPU oracle for the batched stiff-chemistry integrator.
//
// TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke entry point and the
// CPU-baseline leg of the benchmark load this library. The GPU path neither
// links nor calls it, and this file includes nothing from the GPU path.
//
// Plain, slow, FP64 restatement of what the method computes for one cell
// (paper: Introduction, composition vector and f = dphi/dt; Methodology,
// "Analytical Jacobian and improved ODE solution": analytical J_ij = df_i/dphi_j,
// LU decomposition and back substitution inside an implicit ODE solver). The
// paper prints no formulas beyond those definitions, so the kinetics below are
// the textbook constant-pressure adiabatic finite-rate model:
//   * NASA 7-coefficient polynomials for cp/R, H/RT, S/R.
//   * kf = A T^b exp(-Ea_R/T); Kc = exp(-dG/RT) (P0/(Rc T))^dnu; kr = kf/Kc.
//   * third-body [M] = sum eps_k C_k; Lindemann and Troe falloff (the
//     Gilbert-Luther-Troe broadening as given in the Chemkin theory manual).
//   * y = [T, Y_1..Y_K]; C_k = rho Y_k/W_k; rho = p Wbar/(Rc T);
//     dY_k/dt = W_k omega_k/rho; dT/dt = -sum_k h_k omega_k/(rho cp).
//   * Rosenbrock method RODAS4 (Hairer & Wanner, Solving ODEs II, Sec. VI.4)
//     in its original form (I - h gamma J) k_i = h f(y0 + sum a_ij k_j)
//     + h J sum g_ij k_j (Sec. IV.7, Eq. 7.4), WRMS error norm, standard
//     step-size controller, Hairer-Wanner starting step (Solving ODEs I,
//     Sec. II.4), temperature recovery from the conserved mass enthalpy.
//
// Compiled with -ffp-contract=off so results do not depend on FMA contraction.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kRc = 8.31446261815324e7;  // erg / (mol K)
const double kP0 = 1.01325e6;           // dyn / cm^2 (standard state, 1 atm)

}  // namespace

extern "C" {

// Mechanism arrays, same meaning and layout as the synthetic generator's arrays.
struct OMech {
  int32_t K, I, E;
  const double* W;          // [K]
  const int32_t* elem;      // [K][E]
  const double* nasa_lo;    // [K][7]
  const double* nasa_hi;    // [K][7]
  const double* T_lo;       // [K]
  const double* T_mid;      // [K]
  const double* T_hi;       // [K]
  const int32_t* rxn_type;  // [I] 0 elementary, 1 third body, 2 Lindemann, 3 Troe
  const int32_t* reac_idx;  // [I][2]
  const int32_t* reac_nu;   // [I][2]
  const int32_t* prod_idx;  // [I][2]
  const int32_t* prod_nu;   // [I][2]
  const int32_t* reversible;  // [I]
  const double* A;          // [I]
  const double* b;          // [I]
  const double* Ea_R;       // [I]
  const double* A0;         // [I]
  const double* b0;         // [I]
  const double* Ea0_R;      // [I]
  const double* troe;       // [I][4] alpha, T***, T*, T**
  const double* eff;        // [I][K]
};

}  // extern "C"

namespace {

inline double re(double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

template <class S>
S ipow(const S& x, int n) {
  S r = S(1.0);
  for (int i = 0; i < n; ++i) r = r * x;
  return r;
}

// ---------------------------------------------------------------- thermo
// NASA-7: cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
//         H/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
//         S/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
template <class S>
void thermo_species(const OMech& m, int k, const S& T, S& cp_R, S& h_RT, S& s_R) {
  const double* a = (re(T) < m.T_mid[k]) ? &m.nasa_lo[7 * k] : &m.nasa_hi[7 * k];
  S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
  cp_R = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
  h_RT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
  s_R = a[0] * std::log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
}

// d(cp/R)/dT
double dcp_R_dT(const OMech& m, int k, double T) {
  const double* a = (T < m.T_mid[k]) ? &m.nasa_lo[7 * k] : &m.nasa_hi[7 * k];
  return a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T;
}

// ---------------------------------------------------------------- rates
// Rates of progress q_i for temperature T and concentrations C (mol/cm^3).
// Also returns the forward and reverse rate coefficients actually applied
// (for falloff reactions, k = k_inf Pr/(1+Pr) F; for third-body reactions the
// [M] factor multiplies q, not kf).
template <class S>
void rates(const OMech& m, const S& T, const S* C, S* kf_out, S* kr_out, S* q_out) {
  const int K = m.K, I = m.I;
  std::vector<S> g_RT(K);
  for (int k = 0; k < K; ++k) {
    S cp, h, s;
    thermo_species(m, k, T, cp, h, s);
    g_RT[k] = h - s;
  }
  S logT = std::log(T);
  for (int i = 0; i < I; ++i) {
    const int type = m.rxn_type[i];
    S kinf = std::exp(std::log(m.A[i]) + m.b[i] * logT - m.Ea_R[i] / T);
    S kf = kinf;
    S Mconc = S(0.0);
    if (type != 0) {
      for (int k = 0; k < K; ++k) Mconc = Mconc + m.eff[(size_t)i * K + k] * C[k];
    }
    if (type == 2 || type == 3) {
      S k0 = std::exp(std::log(m.A0[i]) + m.b0[i] * logT - m.Ea0_R[i] / T);
      S Pr = k0 * Mconc / kinf;
      S F = S(1.0);
      if (type == 3) {
        const double* tr = &m.troe[4 * i];
        S Fcent = (1.0 - tr[0]) * std::exp(-T / tr[1]) + tr[0] * std::exp(-T / tr[2]);
        if (tr[3] > 0.0) Fcent = Fcent + std::exp(-tr[3] / T);
        S lF = std::log10(Fcent);
        S c = -0.4 - 0.67 * lF;
        S nn = 0.75 - 1.27 * lF;
        S x = std::log10(Pr) + c;
        S f1 = x / (nn - 0.14 * x);
        S lgF = lF / (1.0 + f1 * f1);
        F = std::pow(S(10.0), lgF);
      }
      kf = kinf * (Pr / (1.0 + Pr)) * F;
    }
    // Equilibrium constant from the Gibbs energies.
    S dG = S(0.0);
    int dnu = 0;
    for (int s = 0; s < 2; ++s) {
      if (m.prod_idx[2 * i + s] >= 0) {
        dG = dG + (double)m.prod_nu[2 * i + s] * g_RT[m.prod_idx[2 * i + s]];
        dnu += m.prod_nu[2 * i + s];
      }
      if (m.reac_idx[2 * i + s] >= 0) {
        dG = dG - (double)m.reac_nu[2 * i + s] * g_RT[m.reac_idx[2 * i + s]];
        dnu -= m.reac_nu[2 * i + s];
      }
    }
    S Kc = std::exp(-dG);
    if (dnu > 0) Kc = Kc * ipow(S(kP0) / (kRc * T), dnu);
    if (dnu < 0) Kc = Kc / ipow(S(kP0) / (kRc * T), -dnu);
    S kr = m.reversible[i] ? kf / Kc : S(0.0);
    S Pf = S(1.0), Pb = S(1.0);
    for (int s = 0; s < 2; ++s) {
      if (m.reac_idx[2 * i + s] >= 0) Pf = Pf * ipow(C[m.reac_idx[2 * i + s]], m.reac_nu[2 * i + s]);
      if (m.prod_idx[2 * i + s] >= 0) Pb = Pb * ipow(C[m.prod_idx[2 * i + s]], m.prod_nu[2 * i + s]);
    }
    S q = kf * Pf - kr * Pb;
    if (type == 1) q = q * Mconc;
    if (kf_out) kf_out[i] = kf;
    if (kr_out) kr_out[i] = kr;
    q_out[i] = q;
  }
}

// Net stoichiometric coefficient of species k in reaction i.
int nu_net(const OMech& m, int k, int i) {
  int v = 0;
  for (int s = 0; s < 2; ++s) {
    if (m.prod_idx[2 * i + s] == k) v += m.prod_nu[2 * i + s];
    if (m.reac_idx[2 * i + s] == k) v -= m.reac_nu[2 * i + s];
  }
  return v;
}

// ---------------------------------------------------------------- RHS
// y = [T, Y_1..Y_K], constant pressure p, adiabatic.
template <class S>
void rhs(const OMech& m, double p, const S* y, S* f) {
  const int K = m.K, I = m.I;
  S T = y[0];
  S sumYW = S(0.0);
  for (int k = 0; k < K; ++k) sumYW = sumYW + y[1 + k] / m.W[k];
  S rho = p / (kRc * T * sumYW);
  std::vector<S> C(K), q(I), omega(K, S(0.0));
  for (int k = 0; k < K; ++k) C[k] = rho * y[1 + k] / m.W[k];
  rates(m, T, C.data(), (S*)nullptr, (S*)nullptr, q.data());
  for (int i = 0; i < I; ++i) {
    for (int k = 0; k < K; ++k) {
      int v = nu_net(m, k, i);
      if (v != 0) omega[k] = omega[k] + (double)v * q[i];
    }
  }
  S cp_mass = S(0.0), Qh = S(0.0);
  for (int k = 0; k < K; ++k) {
    S cp, h, s;
    thermo_species(m, k, T, cp, h, s);
    cp_mass = cp_mass + y[1 + k] * cp * kRc / m.W[k];
    Qh = Qh + h * kRc * T * omega[k];
  }
  f[0] = -Qh / (rho * cp_mass);
  for (int k = 0; k < K; ++k) f[1 + k] = m.W[k] * omega[k] / rho;
}

// ---------------------------------------------------------------- analytic Jacobian
// Dense chain rule written out from the RHS definitions. J row-major n x n, n = K+1.
void jac_analytic(const OMech& m, double p, const double* y, double* J, double* f_out) {
  const int K = m.K, I = m.I, n = K + 1;
  const double T = y[0];
  std::vector<double> cp_R(K), h_RT(K), s_R(K), dcp(K);
  for (int k = 0; k < K; ++k) {
    thermo_species(m, k, T, cp_R[k], h_RT[k], s_R[k]);
    dcp[k] = dcp_R_dT(m, k, T);
  }
  double sumYW = 0.0;
  for (int k = 0; k < K; ++k) sumYW += y[1 + k] / m.W[k];
  const double Wbar = 1.0 / sumYW;
  const double rho = p / (kRc * T * sumYW);
  std::vector<double> C(K);
  for (int k = 0; k < K; ++k) C[k] = rho * y[1 + k] / m.W[k];
  // dC_k/dY_j and dC_k/dT
  std::vector<double> dCdY((size_t)K * K), dCdT(K);
  for (int k = 0; k < K; ++k) {
    dCdT[k] = -C[k] / T;
    for (int j = 0; j < K; ++j)
      dCdY[(size_t)k * K + j] = (k == j ? rho / m.W[k] : 0.0) - C[k] * Wbar / m.W[j];
  }
  // per-reaction partials at fixed C
  std::vector<double> q(I), dqdT(I), dqdC((size_t)I * K, 0.0);
  const double logT = std::log(T);
  for (int i = 0; i < I; ++i) {
    const int type = m.rxn_type[i];
    double kinf = std::exp(std::log(m.A[i]) + m.b[i] * logT - m.Ea_R[i] / T);
    double dlnkinf = m.b[i] / T + m.Ea_R[i] / (T * T);
    double dG = 0.0, dH = 0.0;
    int dnu = 0;
    for (int s = 0; s < 2; ++s) {
      int kp = m.prod_idx[2 * i + s], kr_ = m.reac_idx[2 * i + s];
      if (kp >= 0) {
        dG += m.prod_nu[2 * i + s] * (h_RT[kp] - s_R[kp]);
        dH += m.prod_nu[2 * i + s] * h_RT[kp];
        dnu += m.prod_nu[2 * i + s];
      }
      if (kr_ >= 0) {
        dG -= m.reac_nu[2 * i + s] * (h_RT[kr_] - s_R[kr_]);
        dH -= m.reac_nu[2 * i + s] * h_RT[kr_];
        dnu -= m.reac_nu[2 * i + s];
      }
    }
    double Kc = std::exp(-dG) * std::pow(kP0 / (kRc * T), (double)dnu);
    // d ln Kc / dT = dH/(R T^2) - dnu/T, with dH/(RT) = dH here.
    double dlnKc = dH / T - dnu / T;
    double Mconc = 0.0;
    if (type != 0)
      for (int k = 0; k < K; ++k) Mconc += m.eff[(size_t)i * K + k] * C[k];
    // forward products and their derivatives
    double Pf = 1.0, Pb = 1.0;
    std::vector<double> dPf(K, 0.0), dPb(K, 0.0);
    for (int s = 0; s < 2; ++s) {
      if (m.reac_idx[2 * i + s] >= 0) Pf *= ipow(C[m.reac_idx[2 * i + s]], m.reac_nu[2 * i + s]);
      if (m.prod_idx[2 * i + s] >= 0) Pb *= ipow(C[m.prod_idx[2 * i + s]], m.prod_nu[2 * i + s]);
    }
    for (int s = 0; s < 2; ++s) {
      int kk = m.reac_idx[2 * i + s];
      if (kk >= 0) {
        double d = m.reac_nu[2 * i + s] * ipow(C[kk], m.reac_nu[2 * i + s] - 1);
        int o = m.reac_idx[2 * i + (1 - s)];
        if (o >= 0) d *= ipow(C[o], m.reac_nu[2 * i + (1 - s)]);
        dPf[kk] += d;
      }
      kk = m.prod_idx[2 * i + s];
      if (kk >= 0) {
        double d = m.prod_nu[2 * i + s] * ipow(C[kk], m.prod_nu[2 * i + s] - 1);
        int o = m.prod_idx[2 * i + (1 - s)];
        if (o >= 0) d *= ipow(C[o], m.prod_nu[2 * i + (1 - s)]);
        dPb[kk] += d;
      }
    }
    double* dq = &dqdC[(size_t)i * K];
    const bool rev = m.reversible[i] != 0;
    if (type == 0 || type == 1) {
      double kf = kinf, dkf = kinf * dlnkinf;
      double kr = rev ? kf / Kc : 0.0;
      double dkr = rev ? kr * (dlnkinf - dlnKc) : 0.0;
      double base = kf * Pf - kr * Pb;
      double Mf = (type == 1) ? Mconc : 1.0;
      q[i] = Mf * base;
      dqdT[i] = Mf * (dkf * Pf - dkr * Pb);
      for (int j = 0; j < K; ++j) {
        dq[j] = Mf * (kf * dPf[j] - kr * dPb[j]);
        if (type == 1) dq[j] += m.eff[(size_t)i * K + j] * base;
      }
    } else {
      double k0 = std::exp(std::log(m.A0[i]) + m.b0[i] * logT - m.Ea0_R[i] / T);
      double dlnk0 = m.b0[i] / T + m.Ea0_R[i] / (T * T);
      double Pr = k0 * Mconc / kinf;
      double dPr_dM = k0 / kinf;
      double dPr_dT = Pr * (dlnk0 - dlnkinf);
      double F = 1.0, dF_dPr = 0.0, dF_dT = 0.0;
      if (type == 3) {
        const double* tr = &m.troe[4 * i];
        double e3 = std::exp(-T / tr[1]), e1 = std::exp(-T / tr[2]);
        double Fcent = (1.0 - tr[0]) * e3 + tr[0] * e1;
        double dFcent = -(1.0 - tr[0]) / tr[1] * e3 - tr[0] / tr[2] * e1;
        if (tr[3] > 0.0) {
          double e2 = std::exp(-tr[3] / T);
          Fcent += e2;
          dFcent += tr[3] / (T * T) * e2;
        }
        const double ln10 = std::log(10.0);
        double lF = std::log10(Fcent);
        double dlF_dT = dFcent / (Fcent * ln10);
        double c = -0.4 - 0.67 * lF, nn = 0.75 - 1.27 * lF;
        double L = std::log10(Pr);
        double x = L + c;
        double den = nn - 0.14 * x;
        double f1 = x / den;
        double g = 1.0 + f1 * f1;
        double lgF = lF / g;
        F = std::pow(10.0, lgF);
        // partials of f1
        double df1_dL = nn / (den * den);
        double dx_dlF = -0.67, dden_dlF = -1.27 + 0.14 * 0.67;
        double df1_dlF = (dx_dlF * den - x * dden_dlF) / (den * den);
        double dlgF_dL = -lF * 2.0 * f1 / (g * g) * df1_dL;
        double dlgF_dlF = 1.0 / g - lF * 2.0 * f1 / (g * g) * df1_dlF;
        dF_dPr = F * ln10 * dlgF_dL / (Pr * ln10);
        dF_dT = F * ln10 * dlgF_dlF * dlF_dT;  // at fixed Pr
      }
      double kfo = kinf * Pr / (1.0 + Pr) * F;
      double dk_dM = kinf * F / ((1.0 + Pr) * (1.0 + Pr)) * dPr_dM + kinf * Pr / (1.0 + Pr) * dF_dPr * dPr_dM;
      double dk_dT = kinf * dlnkinf * Pr / (1.0 + Pr) * F + kinf * F / ((1.0 + Pr) * (1.0 + Pr)) * dPr_dT +
                     kinf * Pr / (1.0 + Pr) * (dF_dT + dF_dPr * dPr_dT);
      double kr = rev ? kfo / Kc : 0.0;
      double net = Pf - (rev ? Pb / Kc : 0.0);
      q[i] = kfo * Pf - kr * Pb;
      dqdT[i] = dk_dT * net + (rev ? kfo * Pb / Kc * dlnKc : 0.0);
      for (int j = 0; j < K; ++j)
        dq[j] = kfo * dPf[j] - kr * dPb[j] + m.eff[(size_t)i * K + j] * dk_dM * net;
    }
  }
  // dq_i/dY_j and total dq_i/dT
  std::vector<double> dqdY((size_t)I * K, 0.0), dqdTt(I);
  for (int i = 0; i < I; ++i) {
    double t = dqdT[i];
    for (int l = 0; l < K; ++l) t += dqdC[(size_t)i * K + l] * dCdT[l];
    dqdTt[i] = t;
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
      for (int l = 0; l < K; ++l) s += dqdC[(size_t)i * K + l] * dCdY[(size_t)l * K + j];
      dqdY[(size_t)i * K + j] = s;
    }
  }
  // production rates and partials
  std::vector<double> omega(K, 0.0), domdT(K, 0.0), domdY((size_t)K * K, 0.0);
  for (int i = 0; i < I; ++i)
    for (int k = 0; k < K; ++k) {
      int v = nu_net(m, k, i);
      if (v == 0) continue;
      omega[k] += v * q[i];
      domdT[k] += v * dqdTt[i];
      for (int j = 0; j < K; ++j) domdY[(size_t)k * K + j] += v * dqdY[(size_t)i * K + j];
    }
  // species rows: f_k = W_k omega_k / rho
  const double drho_dT = -rho / T;
  std::vector<double> f(n);
  for (int k = 0; k < K; ++k) {
    f[1 + k] = m.W[k] * omega[k] / rho;
    J[(size_t)(1 + k) * n + 0] = m.W[k] * domdT[k] / rho - m.W[k] * omega[k] * drho_dT / (rho * rho);
    for (int j = 0; j < K; ++j) {
      double drho_dY = -rho * Wbar / m.W[j];
      J[(size_t)(1 + k) * n + 1 + j] =
          m.W[k] * domdY[(size_t)k * K + j] / rho - m.W[k] * omega[k] * drho_dY / (rho * rho);
    }
  }
  // temperature row: f_T = -Qh / (rho cpm)
  double cpm = 0.0, dcpm_dT = 0.0, Qh = 0.0, dQh_dT = 0.0;
  for (int k = 0; k < K; ++k) {
    cpm += y[1 + k] * cp_R[k] * kRc / m.W[k];
    dcpm_dT += y[1 + k] * dcp[k] * kRc / m.W[k];
    double hmol = h_RT[k] * kRc * T;
    Qh += hmol * omega[k];
    dQh_dT += cp_R[k] * kRc * omega[k] + hmol * domdT[k];
  }
  f[0] = -Qh / (rho * cpm);
  const double den = rho * cpm;
  J[0] = -dQh_dT / den + Qh / (den * den) * (drho_dT * cpm + rho * dcpm_dT);
  for (int j = 0; j < K; ++j) {
    double dQh = 0.0;
    for (int k = 0; k < K; ++k) dQh += h_RT[k] * kRc * T * domdY[(size_t)k * K + j];
    double drho_dY = -rho * Wbar / m.W[j];
    double dcpm = cp_R[j] * kRc / m.W[j];
    J[1 + j] = -dQh / den + Qh / (den * den) * (drho_dY * cpm + rho * dcpm);
  }
  if (f_out)
    for (int i = 0; i < n; ++i) f_out[i] = f[i];
}

// ---------------------------------------------------------------- dense LU
// Doolittle LU with partial pivoting (row swap to the largest |a_ik|; the
// lowest row index wins ties), in place, row-major. Returns 0 or 1+k for a
// zero pivot at column k.
int lu_factor(int n, double* a, int32_t* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(a[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      a[(size_t)i * n + k] /= a[(size_t)k * n + k];
      double l = a[(size_t)i * n + k];
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void lu_solve(int n, const double* a, const int32_t* piv, double* x) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(x[k], x[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
    x[i] /= a[(size_t)i * n + i];
  }
}

// ---------------------------------------------------------------- tableaus
// A Rosenbrock method in its original form (Hairer & Wanner II, Sec. IV.7, Eq. 7.1):
//   (I - h gamma W) k_i = h f(y0 + sum_{j<i} alpha_ij k_j) + h W sum_{j<i} gamma_ij k_j,
//   y1 = y0 + sum b_i k_i, embedded yhat = y0 + sum bhat_i k_i,
// with W the Jacobian (Rosenbrock / ROW methods) or any approximation of it (W-methods).
// q = order of the embedded solution + 1, the exponent of the step-size control.
struct Tableau {
  int s;
  double alpha[6][6];
  double gam[6][6];  // Gamma, lower triangular including the diagonal gamma
  double b[6], bhat[6];
  double gamma, q;
};

// RODAS4, Hairer & Wanner, Solving ODEs II, Sec. VI.4: the published coefficients
// in the transformed variables u_i = sum_j gamma_ij k_j (Sec. IV.7, Eq. 7.3):
// a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b^T Gamma^-1. The
// original (alpha, gamma, b, bhat) form the oracle integrates with is
// recovered here by inverting that transformation.
Tableau make_rodas4() {
  const double g = 0.25;
  double A[6][6] = {{0}};
  double Cc[6][6] = {{0}};
  A[1][0] = 1.544;
  A[2][0] = 0.9466785280815826;
  A[2][1] = 0.2557011698983284;
  A[3][0] = 3.314825187068521;
  A[3][1] = 2.896124015972201;
  A[3][2] = 0.9986419139977817;
  A[4][0] = 1.221224509226641;
  A[4][1] = 6.019134481288629;
  A[4][2] = 12.53708332932087;
  A[4][3] = -0.687886036105895;
  for (int j = 0; j < 4; ++j) A[5][j] = A[4][j];
  A[5][4] = 1.0;
  Cc[1][0] = -5.6688;
  Cc[2][0] = -2.430093356833875;
  Cc[2][1] = -0.2063599157091915;
  Cc[3][0] = -0.1073529058151375;
  Cc[3][1] = -9.594562251023355;
  Cc[3][2] = -20.47028614809616;
  Cc[4][0] = 7.496443313967647;
  Cc[4][1] = -10.24680431464352;
  Cc[4][2] = -33.99990352819905;
  Cc[4][3] = 11.7089089320616;
  Cc[5][0] = 8.083246795921522;
  Cc[5][1] = -7.981132988064893;
  Cc[5][2] = -31.52159432874371;
  Cc[5][3] = 16.31930543123136;
  Cc[5][4] = -6.058818238834054;
  double mm[6] = {A[4][0], A[4][1], A[4][2], A[4][3], 1.0, 1.0};
  double mh[6] = {A[4][0], A[4][1], A[4][2], A[4][3], 1.0, 0.0};
  // Gamma^-1 = diag(1/g) - C ; invert the lower triangular matrix.
  double Gi[6][6] = {{0}}, G[6][6] = {{0}};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Gi[i][j] = (i == j ? 1.0 / g : 0.0) - Cc[i][j];
  for (int j = 0; j < 6; ++j) {
    for (int i = 0; i < 6; ++i) {
      if (i < j) { G[i][j] = 0.0; continue; }
      double s = (i == j) ? 1.0 : 0.0;
      for (int l = j; l < i; ++l) s -= Gi[i][l] * G[l][j];
      G[i][j] = s / Gi[i][i];
    }
  }
  Tableau t{};
  t.s = 6;
  t.gamma = g;
  t.q = 4.0;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int l = 0; l < 6; ++l) s += A[i][l] * G[l][j];
      t.alpha[i][j] = (j < i) ? s : 0.0;
      t.gam[i][j] = G[i][j];
    }
  }
  for (int j = 0; j < 6; ++j) {
    double s = 0.0, sh = 0.0;
    for (int l = 0; l < 6; ++l) {
      s += mm[l] * G[l][j];
      sh += mh[l] * G[l][j];
    }
    t.b[j] = s;
    t.bhat[j] = sh;
  }
  return t;
}

// ROS34PW2, J. Rang and L. Angermann, "New Rosenbrock W-methods of order 3 for
// partial differential algebraic equations of index 1", BIT 45 (2005): 4 stages,
// order 3 for ANY W (a W-method), embedded order 2, stiffly accurate, L-stable.
// The published coefficients in the original form.
Tableau make_ros34pw2() {
  const double g = 4.3586652150845900e-01;
  Tableau t{};
  t.s = 4;
  t.gamma = g;
  t.q = 3.0;
  t.alpha[1][0] = 8.7173304301691801e-01;
  t.alpha[2][0] = 8.4457060015369423e-01;
  t.alpha[2][1] = -1.1299064236484185e-01;
  t.alpha[3][2] = 1.0;
  t.gam[1][0] = -8.7173304301691801e-01;
  t.gam[2][0] = -9.0338057013044082e-01;
  t.gam[2][1] = 5.4180672388095326e-02;
  t.gam[3][0] = 2.4212380706095346e-01;
  t.gam[3][1] = -1.2232505839045147e+00;
  t.gam[3][2] = 5.4526025533510214e-01;
  for (int i = 0; i < 4; ++i) t.gam[i][i] = g;
  const double b[4] = {2.4212380706095346e-01, -1.2232505839045147e+00, 1.5452602553351020e+00, g};
  const double bh[4] = {3.7810903145819369e-01, -9.6042292212423178e-02, 0.5, 2.1793326075422950e-01};
  for (int i = 0; i < 4; ++i) {
    t.b[i] = b[i];
    t.bhat[i] = bh[i];
  }
  return t;
}

enum { METHOD_RODAS4 = 0, METHOD_ROS34PW2 = 1 };

const Tableau& tableau(int method = METHOD_RODAS4) {
  static const Tableau t0 = make_rodas4();
  static const Tableau t1 = make_ros34pw2();
  return method == METHOD_ROS34PW2 ? t1 : t0;
}

// ---------------------------------------------------------------- one Rosenbrock step
// Original form (see Tableau) with W = the analytic Jacobian at y0, plus E when E is
// given (a fixed perturbation: the W-method property is that the order survives it).
// Returns 0 on success, nonzero for a singular iteration matrix.
int row_step(const OMech& m, double p, const double* y0, double h, double* y1, double* yhat, int method,
             const double* E) {
  const Tableau& tb = tableau(method);
  const int n = m.K + 1, S = tb.s;
  std::vector<double> J((size_t)n * n), M((size_t)n * n), kst((size_t)S * n), yi(n), fi(n), v(n), Jv(n);
  std::vector<int32_t> piv(n);
  jac_analytic(m, p, y0, J.data(), nullptr);
  if (E)
    for (size_t e = 0; e < (size_t)n * n; ++e) J[e] += E[e];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - h * tb.gamma * J[(size_t)i * n + j];
  if (lu_factor(n, M.data(), piv.data())) return 1;
  for (int s = 0; s < S; ++s) {
    for (int l = 0; l < n; ++l) {
      double a = y0[l], g = 0.0;
      for (int j = 0; j < s; ++j) {
        a += tb.alpha[s][j] * kst[(size_t)j * n + l];
        g += tb.gam[s][j] * kst[(size_t)j * n + l];
      }
      yi[l] = a;
      v[l] = g;
    }
    rhs(m, p, yi.data(), fi.data());
    for (int i = 0; i < n; ++i) {
      double s2 = 0.0;
      for (int j = 0; j < n; ++j) s2 += J[(size_t)i * n + j] * v[j];
      Jv[i] = s2;
    }
    double* ks = &kst[(size_t)s * n];
    for (int i = 0; i < n; ++i) ks[i] = h * fi[i] + h * Jv[i];
    lu_solve(n, M.data(), piv.data(), ks);
  }
  for (int i = 0; i < n; ++i) {
    double a = y0[i], ah = y0[i];
    for (int s = 0; s < S; ++s) {
      a += tb.b[s] * kst[(size_t)s * n + i];
      ah += tb.bhat[s] * kst[(size_t)s * n + i];
    }
    y1[i] = a;
    yhat[i] = ah;
  }
  return 0;
}

int rodas_step(const OMech& m, double p, const double* y0, double h, double* y1, double* yhat) {
  return row_step(m, p, y0, h, y1, yhat, METHOD_RODAS4, nullptr);
}

double wrms(int n, const double* e, const double* ya, const double* yb, double rtol, double atol) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double sc = atol + rtol * std::max(std::fabs(ya[i]), std::fabs(yb[i]));
    double r = e[i] / sc;
    s += r * r;
  }
  return std::sqrt(s / n);
}

// Hairer-Wanner starting step size (Solving ODEs I, Sec. II.4) in the WRMS norm
// with scale atol + rtol |y0_i|; exponent 1/q (embedded order plus one: 1/4 for
// RODAS4, 1/3 for ROS34PW2); clamped to dt. A vanishing derivative selects the
// whole interval.
double h0_estimate(const OMech& m, double p, const double* y0, double dt, double rtol, double atol,
                   double q = 4.0) {
  const int n = m.K + 1;
  std::vector<double> f0(n), f1(n), y1(n), d(n);
  rhs(m, p, y0, f0.data());
  double d0 = wrms(n, y0, y0, y0, rtol, atol);
  double d1 = wrms(n, f0.data(), y0, y0, rtol, atol);
  double ha = (d1 > 1e-300) ? 0.01 * d0 / d1 : dt;
  ha = std::min(ha, dt);
  for (int i = 0; i < n; ++i) y1[i] = y0[i] + ha * f0[i];
  rhs(m, p, y1.data(), f1.data());
  for (int i = 0; i < n; ++i) d[i] = f1[i] - f0[i];
  double d2 = wrms(n, d.data(), y0, y0, rtol, atol) / ha;
  double mx = std::max(d1, d2);
  double hb = (mx > 1e-300) ? std::pow(0.01 / mx, 1.0 / q) : dt;
  return std::min(std::min(100.0 * ha, hb), dt);
}

double enthalpy_mass(const OMech& m, double T, const double* Y) {
  double h = 0.0;
  for (int k = 0; k < m.K; ++k) {
    double cp, hr, s;
    thermo_species(m, k, T, cp, hr, s);
    h += Y[k] * hr * kRc * T / m.W[k];
  }
  return h;
}

double cp_mass(const OMech& m, double T, const double* Y) {
  double c = 0.0;
  for (int k = 0; k < m.K; ++k) {
    double cp, hr, s;
    thermo_species(m, k, T, cp, hr, s);
    c += Y[k] * cp * kRc / m.W[k];
  }
  return c;
}

// Newton solve of h(T, Y) = h_target from T_guess; |dT| < 1e-10 T.
double recover_T(const OMech& m, const double* Y, double h_target, double T_guess) {
  double T = T_guess;
  for (int it = 0; it < 50; ++it) {
    double dT = (enthalpy_mass(m, T, Y) - h_target) / cp_mass(m, T, Y);
    T -= dT;
    if (std::fabs(dT) < 1e-10 * T) break;
  }
  return T;
}

enum { ST_OK = 0, ST_MAX_STEPS = 1, ST_H_UNDERFLOW = 2, ST_NONFINITE = 3, ST_T_RANGE = 4 };

struct CellResult {
  int substeps, rejects, status;
  double h_first, T_ode;
};

// Adaptive integration of one cell over [0, dt]; y in/out (last accepted state).
CellResult integrate_cell(const OMech& m, double p, double* y, double dt, double rtol, double atol,
                          int max_steps, double h_init, int method) {
  const int n = m.K + 1;
  const double q = tableau(method).q;
  const double facmin = 0.2, facmax = 5.0, safety = 0.9, h_min = 1e-20;
  CellResult r{0, 0, ST_OK, 0.0, y[0]};
  std::vector<double> y1(n), yh(n), e(n);
  const double h_target = enthalpy_mass(m, y[0], y + 1);
  double h = (h_init > 0.0) ? std::min(h_init, dt) : h0_estimate(m, p, y, dt, rtol, atol, q);
  double t = 0.0;
  bool after_reject = false;
  while (true) {
    if (dt - t <= 1e-12 * dt) break;
    if (r.substeps >= max_steps) { r.status = ST_MAX_STEPS; break; }
    if (!(h >= h_min)) { r.status = ST_H_UNDERFLOW; break; }
    if (t + h > dt) h = dt - t;
    int bad = row_step(m, p, y, h, y1.data(), yh.data(), method, nullptr);
    r.substeps++;
    double err;
    bool finite = !bad;
    for (int i = 0; i < n && finite; ++i) finite = std::isfinite(y1[i]) && std::isfinite(yh[i]);
    if (finite) {
      for (int i = 0; i < n; ++i) e[i] = y1[i] - yh[i];
      err = wrms(n, e.data(), y, y1.data(), rtol, atol);
      if (!std::isfinite(err)) finite = false;
    }
    if (!finite) {
      r.rejects++;
      after_reject = true;
      h *= facmin;
      continue;
    }
    double fac = (err > 0.0) ? safety * std::pow(err, -1.0 / q) : facmax;
    if (err <= 1.0) {
      t += h;
      for (int i = 0; i < n; ++i) y[i] = y1[i];
      if (r.h_first == 0.0) r.h_first = h;
      fac = std::min(std::max(fac, facmin), after_reject ? 1.0 : facmax);
      after_reject = false;
      h *= fac;
    } else {
      r.rejects++;
      after_reject = true;
      h *= std::max(fac, facmin);
    }
  }
  r.T_ode = y[0];
  if (r.status == ST_OK) {
    y[0] = recover_T(m, y + 1, h_target, y[0]);
    if (!(y[0] >= 200.0 && y[0] <= 6000.0)) r.status = ST_T_RANGE;
  }
  return r;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void oracle_thermo(const OMech* m, double T, double* cp_R, double* h_RT, double* s_R) {
  for (int k = 0; k < m->K; ++k) thermo_species(*m, k, T, cp_R[k], h_RT[k], s_R[k]);
}

// Rate coefficients and rates of progress at state y = [T, Y].
void oracle_rates(const OMech* m, double p, const double* y, double* kf, double* kr, double* q) {
  const int K = m->K;
  double sumYW = 0.0;
  for (int k = 0; k < K; ++k) sumYW += y[1 + k] / m->W[k];
  double rho = p / (kRc * y[0] * sumYW);
  std::vector<double> C(K);
  for (int k = 0; k < K; ++k) C[k] = rho * y[1 + k] / m->W[k];
  rates(*m, y[0], C.data(), kf, kr, q);
}

// Rates of progress at temperature T and given concentrations (mol/cm^3).
void oracle_rates_conc(const OMech* m, double T, const double* C, double* kf, double* kr, double* q) {
  rates(*m, T, C, kf, kr, q);
}

void oracle_rhs(const OMech* m, double p, const double* y, double* f) { rhs(*m, p, y, f); }

void oracle_jac(const OMech* m, double p, const double* y, double* J) {
  jac_analytic(*m, p, y, J, nullptr);
}

// Central finite differences with step rel * max(|y_j|, floor).
void oracle_jac_fd(const OMech* m, double p, const double* y, double* J, double rel, double floor) {
  const int n = m->K + 1;
  std::vector<double> yp(y, y + n), ym(y, y + n), fp(n), fm(n);
  for (int j = 0; j < n; ++j) {
    double d = rel * std::max(std::fabs(y[j]), floor);
    yp[j] = y[j] + d;
    ym[j] = y[j] - d;
    rhs(*m, p, yp.data(), fp.data());
    rhs(*m, p, ym.data(), fm.data());
    for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = (fp[i] - fm[i]) / (yp[j] - ym[j]);
    yp[j] = y[j];
    ym[j] = y[j];
  }
}

// Complex-step derivative: J_ij = Im f_i(y + i h e_j) / h, h = 1e-30.
void oracle_jac_cstep(const OMech* m, double p, const double* y, double* J) {
  const int n = m->K + 1;
  const double hs = 1e-30;
  std::vector<std::complex<double>> yc(n), fc(n);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) yc[i] = std::complex<double>(y[i], i == j ? hs : 0.0);
    rhs(*m, p, yc.data(), fc.data());
    for (int i = 0; i < n; ++i) J[(size_t)i * n + j] = fc[i].imag() / hs;
  }
}

int oracle_lu_factor(int n, double* a, int32_t* piv) { return lu_factor(n, a, piv); }
void oracle_lu_solve(int n, const double* a, const int32_t* piv, double* x) { lu_solve(n, a, piv, x); }

// Tableau of `method` (0 RODAS4, 1 ROS34PW2): alpha[36], gamma[36] (row-major 6x6,
// Gamma including its diagonal, zero beyond the stage count), b[6], bhat[6];
// returns the number of stages.
int oracle_tableau_m(int method, double* alpha, double* gam, double* b, double* bhat, double* q) {
  const Tableau& t = tableau(method);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      alpha[6 * i + j] = t.alpha[i][j];
      gam[6 * i + j] = t.gam[i][j];
    }
  for (int i = 0; i < 6; ++i) {
    b[i] = t.b[i];
    bhat[i] = t.bhat[i];
  }
  if (q) *q = t.q;
  return t.s;
}

void oracle_tableau(double* alpha, double* gam, double* b, double* bhat) {
  oracle_tableau_m(METHOD_RODAS4, alpha, gam, b, bhat, nullptr);
}

int oracle_rodas_step(const OMech* m, double p, const double* y0, double h, double* y1, double* yhat) {
  return rodas_step(*m, p, y0, h, y1, yhat);
}

// One step of `method` with W = J(y0) + E (E nullable: the exact Jacobian).
int oracle_row_step(const OMech* m, double p, const double* y0, double h, double* y1, double* yhat, int method,
                    const double* E) {
  return row_step(*m, p, y0, h, y1, yhat, method, E);
}

double oracle_h0(const OMech* m, double p, const double* y0, double dt, double rtol, double atol) {
  return h0_estimate(*m, p, y0, dt, rtol, atol);
}

double oracle_h0_m(const OMech* m, double p, const double* y0, double dt, double rtol, double atol, int method) {
  return h0_estimate(*m, p, y0, dt, rtol, atol, tableau(method).q);
}

double oracle_enthalpy_mass(const OMech* m, double T, const double* Y) { return enthalpy_mass(*m, T, Y); }

double oracle_recover_T(const OMech* m, const double* Y, double h_target, double T_guess) {
  return recover_T(*m, Y, h_target, T_guess);
}

// Integrate n cells over dt with `method` (0 RODAS4, 1 ROS34PW2; W = the analytic
// Jacobian). T[n] and Y[n][K] in/out, p[n] in. h0 (nullable): per-cell initial
// step; <= 0 or NULL selects the starting-step heuristic. Per-cell outputs are
// nullable. Returns the number of cells with status != 0.
int64_t oracle_integrate(const OMech* m, int64_t n_cells, double* T, const double* p, double* Y,
                         double dt, double rtol, double atol, int32_t max_steps, const double* h0,
                         int32_t* substeps, int32_t* rejects, double* h_first, int32_t* status,
                         double* T_ode, int32_t n_threads, int32_t method) {
  const int K = m->K;
  int64_t failed = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : failed)
#endif
  for (int64_t c = 0; c < n_cells; ++c) {
    std::vector<double> y(K + 1);
    y[0] = T[c];
    for (int k = 0; k < K; ++k) y[1 + k] = Y[(size_t)c * K + k];
    double hi = h0 ? h0[c] : 0.0;
    CellResult r = integrate_cell(*m, p[c], y.data(), dt, rtol, atol, max_steps, hi, method);
    T[c] = y[0];
    for (int k = 0; k < K; ++k) Y[(size_t)c * K + k] = y[1 + k];
    if (substeps) substeps[c] = r.substeps;
    if (rejects) rejects[c] = r.rejects;
    if (h_first) h_first[c] = r.h_first;
    if (status) status[c] = r.status;
    if (T_ode) T_ode[c] = r.T_ode;
    if (r.status != ST_OK) failed += 1;
  }
  return failed;
}

int oracle_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
