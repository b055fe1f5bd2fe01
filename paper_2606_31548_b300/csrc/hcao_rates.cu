// hcao_rates.cu -- host code: the thermal dissociation probability P(T) of
// Eq. recomb-correct and the partition sums behind K_eq, for the rate tables
// of the recombination reactions.
//
// P(T) = (1/Z) sum over all level combinations s of exp(-X_s/kT) Q(a, max(0,
// (Dx - X_s)/kT)), X_s the excitation above the ground state and Dx the
// threshold above it.  Modes with identical level lists (the C-H stretches of
// a methane-like molecule, degenerate bends) are summed as groups: a group of
// m identical modes is enumerated as multisets of levels with their
// multiplicities m!/prod(c!), so a 4 + 3 + 2 mode molecule needs ~1e4-1e5
// terms per temperature instead of ~1e7 ordered tuples.  Every term is
// positive: states at or above the threshold (Q = 1) are summed through
// suffix and tail sums of the groups' Boltzmann factors, never as a partition
// sum minus the states below it.
#include "hcao_rates.h"

#include <algorithm>
#include <cmath>

namespace hcao {

double rec_node_T(int i) { return 500.0 * std::pow(2.0, (double)i / 32.0); }

// Q(a, x): series of the lower function P(a, x) = x^a e^-x / Gamma(a+1) *
// sum_n x^n / ((a+1)...(a+n)) when x < a + 1, else the continued fraction
// Gamma(a, x) = e^-x x^a / (x + 1 - a - 1(1-a)/(x + 3 - a - 2(2-a)/(x + 5 - a - ...)))
// evaluated from the top down in the modified Lentz form.
double inc_gamma_q(double a, double x) {
    if (!(x > 0.0)) return 1.0;
    const double lfac = a * std::log(x) - x - std::lgamma(a);
    if (x < a + 1.0) {
        double t = 1.0 / a, s = t;
        for (int n = 1; n < 100000; ++n) {
            t = t * x / (a + n);
            s += t;
            if (t < s * 1e-17) break;
        }
        return 1.0 - s * std::exp(lfac);
    }
    const double eps = 1e-300;
    double bn = x + 1.0 - a;
    double f = bn, Cn = bn, Dn = 0.0;
    for (int n = 1; n < 100000; ++n) {
        const double an = -(double)n * ((double)n - a);
        bn += 2.0;
        Dn = bn + an * Dn;
        if (std::fabs(Dn) < eps) Dn = eps;
        Cn = bn + an / Cn;
        if (std::fabs(Cn) < eps) Cn = eps;
        Dn = 1.0 / Dn;
        const double r = Cn * Dn;
        f *= r;
        if (std::fabs(r - 1.0) < 1e-17) break;
    }
    return std::exp(lfac) / f;
}

namespace {

struct Group {
    std::vector<double> x;            // level excitations (ascending)
    int m = 0;                        // identical modes
    std::vector<double> e, w;         // multisets below the threshold: excitation, multiplicity
};

// multisets i_1 <= ... <= i_m of the group's levels with excitation < Dx
void multisets(const Group& g, double Dx, int pos, int from, double X, std::vector<int>& cnt,
               std::vector<std::pair<double, double>>& out) {
    if (pos == g.m) {
        double w = std::tgamma(g.m + 1.0);
        for (int c : cnt)
            if (c > 1) w /= std::tgamma(c + 1.0);
        out.push_back({X, w});
        return;
    }
    for (int i = from; i < (int)g.x.size(); ++i) {
        // every later index is >= i: the smallest completion adds (m - pos) x_i
        if (!(X + (double)(g.m - pos) * g.x[i] < Dx)) break;
        cnt[i]++;
        multisets(g, Dx, pos + 1, i, X + g.x[i], cnt, out);
        cnt[i]--;
    }
}

// sum over ordered tuples of the group's remaining positions whose total
// excitation reaches Dx, of exp(-(X + tuple)/kT); partial X < Dx
double group_tail(const Group& g, const std::vector<double>& bz, const std::vector<double>& suf,
                  double z, double Dx, double kT, int pos, double X) {
    if (pos == g.m) return 0.0;
    double s = 0.0;
    const double zr = std::pow(z, (double)(g.m - pos - 1));
    for (size_t i = 0; i < g.x.size(); ++i) {
        const double Xi = X + g.x[i];
        if (!(Xi < Dx)) {
            s += std::exp(-X / kT) * suf[i] * zr;
            break;
        }
        s += group_tail(g, bz, suf, z, Dx, kT, pos + 1, Xi);
    }
    return s;
}

struct Ctx {
    const std::vector<Group>* G;
    std::vector<std::vector<double>> esuf;  // per group: suffix sums of w exp(-e/kT) over entries
    std::vector<double> tail;                // per group: ordered tuples at or above Dx
    std::vector<double> zrest;               // prod over groups >= g of z^m
    double Dx, kT, a;
};

double walk(const Ctx& c, size_t g, double X, double W) {
    const std::vector<Group>& G = *c.G;
    if (g == G.size()) return W * std::exp(-X / c.kT) * inc_gamma_q(c.a, (c.Dx - X) / c.kT);
    const Group& gr = G[g];
    double s = 0.0;
    for (size_t j = 0; j < gr.e.size(); ++j) {
        const double Xj = X + gr.e[j];
        if (!(Xj < c.Dx)) {
            s += W * std::exp(-X / c.kT) * (c.esuf[g][j] + c.tail[g]) * c.zrest[g + 1];
            return s;
        }
        s += walk(c, g + 1, Xj, W * gr.w[j]);
    }
    s += W * std::exp(-X / c.kT) * c.tail[g] * c.zrest[g + 1];
    return s;
}

std::vector<Group> make_groups(const std::vector<std::vector<double>>& lev, double Dx) {
    std::vector<Group> G;
    std::vector<bool> used(lev.size(), false);
    for (size_t j = 0; j < lev.size(); ++j) {
        if (used[j]) continue;
        Group g;
        for (double E : lev[j]) g.x.push_back(E - lev[j][0]);
        for (size_t k = j; k < lev.size(); ++k)
            if (!used[k] && lev[k] == lev[j]) {
                used[k] = true;
                g.m++;
            }
        std::vector<int> cnt(g.x.size(), 0);
        std::vector<std::pair<double, double>> ms;
        multisets(g, Dx, 0, 0, 0.0, cnt, ms);
        std::sort(ms.begin(), ms.end());
        for (auto& p : ms) {
            g.e.push_back(p.first);
            g.w.push_back(p.second);
        }
        G.push_back(std::move(g));
    }
    return G;
}

}  // namespace

double thermal_diss_prob(const std::vector<std::vector<double>>& lev, double D, double a, double T) {
    double zpe = 0.0;
    for (auto& l : lev) zpe += l[0];
    const double Dx = D - zpe;
    const double kT = 1.380649e-23 * T;
    const std::vector<Group> G = make_groups(lev, Dx);
    Ctx c;
    c.G = &G;
    c.Dx = Dx;
    c.kT = kT;
    c.a = a;
    c.esuf.resize(G.size());
    c.tail.resize(G.size());
    c.zrest.assign(G.size() + 1, 1.0);
    for (size_t g = G.size(); g-- > 0;) {
        const Group& gr = G[g];
        std::vector<double> bz(gr.x.size()), suf(gr.x.size() + 1, 0.0);
        for (size_t i = 0; i < gr.x.size(); ++i) bz[i] = std::exp(-gr.x[i] / kT);
        for (size_t i = gr.x.size(); i-- > 0;) suf[i] = suf[i + 1] + bz[i];
        const double z = suf[0];
        c.zrest[g] = c.zrest[g + 1] * std::pow(z, (double)gr.m);
        c.tail[g] = group_tail(gr, bz, suf, z, Dx, kT, 0, 0.0);
        c.esuf[g].assign(gr.e.size() + 1, 0.0);
        for (size_t j = gr.e.size(); j-- > 0;) c.esuf[g][j] = c.esuf[g][j + 1] + gr.w[j] * std::exp(-gr.e[j] / kT);
    }
    if (!(Dx > 0.0)) return 1.0;
    return walk(c, 0, 0.0, 1.0) / c.zrest[0];
}

// Whitten-Rabinovitch: l oscillators, quanta hnu, E above the ground state.
// With x = E/E_z (E_z = half the sum of the quanta), the correction
// a(x) = 1 - beta w(x), w = 10^(-1.0506 x^(1/4)) for x >= 1 and
// w = 1/(5 x + 2.73 sqrt(x) + 3.51) below, and the WR beta of the paper,
// (l-1)^2 S2 / (l S1^2) with S1 the sum of the quanta and S2 the sum of their
// squares.  The density is
// (E + a E_z)^(l-1) / ((l-1)! prod hnu); computed through its logarithm.
static bool wr_setup(const double* hnu, int l, double& Ez, double& beta, double& lden) {
    if (!hnu || l < 1) return false;
    double s1 = 0.0, s2 = 0.0;
    lden = std::lgamma((double)l);
    for (int k = 0; k < l; ++k) {
        if (!(hnu[k] > 0.0)) return false;
        s1 += hnu[k];
        s2 += hnu[k] * hnu[k];
        lden += std::log(hnu[k]);
    }
    Ez = 0.5 * s1;
    beta = (double)(l - 1) * (double)(l - 1) * s2 / ((double)l * s1 * s1);
    return true;
}

static double wr_log_shape(int l, double Ez, double beta, double E) {
    const double x = E / Ez;
    const double w = x < 1.0 ? 1.0 / (5.0 * x + 2.73 * std::sqrt(x) + 3.51)
                             : std::pow(10.0, -1.0506 * std::sqrt(std::sqrt(x)));
    return (double)(l - 1) * std::log(E + (1.0 - beta * w) * Ez);
}

double wr_density(const double* hnu, int l, double E) {
    double Ez, beta, lden;
    if (!wr_setup(hnu, l, Ez, beta, lden) || !(E >= 0.0)) return NAN;
    return std::exp(wr_log_shape(l, Ez, beta, E) - lden);
}

double wr_diss_prob(const double* hnu, int l, double Dx, double a, double T, int n_samp) {
    double Ez, beta, lden;
    if (!wr_setup(hnu, l, Ez, beta, lden) || n_samp < 1 || !(T > 0.0) || !(a > 0.0)) return NAN;
    if (!(Dx > 0.0)) return 1.0;
    const double kT = 1.380649e-23 * T, dE = Dx / (double)n_samp;
    std::vector<double> lw((size_t)n_samp);
    double top = -INFINITY;
    for (int i = 0; i < n_samp; ++i) {
        const double E = ((double)i + 0.5) * dE;
        lw[(size_t)i] = wr_log_shape(l, Ez, beta, E) - E / kT;
        top = std::max(top, lw[(size_t)i]);
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n_samp; ++i) {
        const double E = ((double)i + 0.5) * dE;
        const double w = std::exp(lw[(size_t)i] - top);
        num += w * inc_gamma_q(a, (Dx - E) / kT);
        den += w;
    }
    return num / den;
}

double zvib_excited(const std::vector<std::vector<double>>& lev, double T) {
    const double kT = 1.380649e-23 * T;
    double z = 1.0;
    for (auto& l : lev) {
        double s = 0.0;
        for (double E : l) s += std::exp(-(E - l[0]) / kT);
        z *= s;
    }
    return z;
}

}  // namespace hcao
