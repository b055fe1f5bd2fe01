// hcao_rates.h -- host-side rate tables of the recombination reactions
// (Sec. "Recombination reactions"): k_r = k_f / K_eq with k_f = P <sigma_T g>,
// P the thermal dissociation probability of Eq. recomb-correct.
#pragma once
#include <vector>

#include "hcao_internal.h"

namespace hcao {

// rate-table node i: T_i = 500 K * 2^(i/32), i < REC_NODES
double rec_node_T(int i);

// Regularised upper incomplete gamma Q(a, x); 1 for x <= 0.
double inc_gamma_q(double a, double x);

// Thermal average, over every combination of the levels of A's modes (lev[j]
// ascending, energies from the well bottom), of Q(a, max(0, (D - E)/kT)).
// D: dissociation threshold from the well bottom, a = 5/2 - omega.
double thermal_diss_prob(const std::vector<std::vector<double>>& lev, double D, double a, double T);

// Whitten-Rabinovitch density of states (1/J) of l oscillators with quanta
// hnu (J) at E (J) above the ground state; NaN for bad arguments.
double wr_density(const double* hnu, int l, double E);

// The sampled (WR) dissociation probability: n_samp midpoint energies below
// the threshold Dx (J above the ground state), weights rho(E) exp(-E/kT),
// P = sum Q(a, (Dx - E)/kT) w / sum w.  NaN for bad arguments.
double wr_diss_prob(const double* hnu, int l, double Dx, double a, double T, int n_samp);

// Vibrational partition sum with energies measured from the ground state.
double zvib_excited(const std::vector<std::vector<double>>& lev, double T);

}  // namespace hcao
