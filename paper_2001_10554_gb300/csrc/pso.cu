// Particle swarm optimisation of QAOA parameters (Section 4, "QAOA with swarm
// particle optimization"): every particle is one virtual quantum device whose
// position theta = (gamma_1..gamma_p, beta_1..beta_p) is scored by the QAOA
// objective L(theta) = <H_MaxCut>, to be maximised.  One swarm step updates
// every velocity from three terms (damping omega, attraction phi_p r_p to the
// particle's own best position, attraction phi_g r_g to the swarm's best),
// moves every particle, and scores all new positions.
//
// The swarms of all graphs of a multi-graph engine step in lockstep: one
// engine call scores the n_graphs x particles positions of a step (state
// g * particles + k is particle k of graph g), so the device sees one batch
// per step however many swarms there are.  The swarm logic itself is this
// host loop; every random number it uses is an input.
#include <cmath>
#include <limits>
#include <vector>

#include "internal.h"

extern "C" {

iqs_status iqs_qaoa_pso(iqs_qaoa* q, int p, int steps, const double* pos0, const double* vel0, const double* rp,
                        const double* rg, double omega, double phi_p, double phi_g, double* trace, double* best_pos,
                        double* best_val) {
  using iqs::report;
  int n = 0, dtype = 0, G = 0, R = 0, ne = 0;
  iqs_status st = iqs_qaoa_info(q, &n, &dtype, &G, &R, &ne);
  if (st != IQS_OK) return st;
  if (p < 1 || p > 64) return report(IQS_EINVAL, "p = %d outside [1, 64]", p);
  if (steps < 0) return report(IQS_EINVAL, "steps must be >= 0");
  if (!pos0 || !vel0 || !trace || !best_pos || !best_val || (steps > 0 && (!rp || !rg)))
    return report(IQS_EINVAL, "an array argument is NULL");
  if (!std::isfinite(omega) || !std::isfinite(phi_p) || !std::isfinite(phi_g))
    return report(IQS_EINVAL, "omega, phi_p and phi_g must be finite");
  const int D = 2 * p;
  const size_t P = (size_t)G * R;
  std::vector<double> x(pos0, pos0 + P * D), v(vel0, vel0 + P * D);
  std::vector<double> pb(x), pval(P), gb((size_t)G * D), gval(G, -std::numeric_limits<double>::infinity());
  std::vector<double> gam(P * p), bet(P * p), L(P), run(G, -std::numeric_limits<double>::infinity());
  for (size_t i = 0; i < P * D; ++i)
    if (!std::isfinite(x[i]) || !std::isfinite(v[i])) return report(IQS_EINVAL, "initial position or velocity not finite");

  auto score = [&]() -> iqs_status {
    for (size_t k = 0; k < P; ++k)
      for (int l = 0; l < p; ++l) {
        gam[k * p + l] = x[k * D + l];
        bet[k * p + l] = x[k * D + p + l];
      }
    return iqs_qaoa_run(q, (int)P, p, gam.data(), bet.data(), L.data(), nullptr, nullptr);
  };
  // best-so-far after each evaluation, particles of a step in order; the
  // swarm's best moves only after the whole step has been scored
  auto record = [&](int step) {
    for (int g = 0; g < G; ++g) {
      double* tr = trace + (size_t)g * (size_t)(steps + 1) * R + (size_t)step * R;
      for (int k = 0; k < R; ++k) {
        const size_t i = (size_t)g * R + k;
        if (L[i] > run[g]) run[g] = L[i];
        tr[k] = run[g];
        if (step == 0 || L[i] > pval[i]) {
          pval[i] = L[i];
          for (int d = 0; d < D; ++d) pb[i * D + d] = x[i * D + d];
        }
      }
      for (int k = 0; k < R; ++k) {
        const size_t i = (size_t)g * R + k;
        if (L[i] > gval[g]) {
          gval[g] = L[i];
          for (int d = 0; d < D; ++d) gb[(size_t)g * D + d] = x[i * D + d];
        }
      }
    }
  };

  if ((st = score()) != IQS_OK) return st;
  record(0);
  for (int s = 1; s <= steps; ++s) {
    for (int g = 0; g < G; ++g)
      for (int k = 0; k < R; ++k) {
        const size_t i = (size_t)g * R + k;
        const double a = phi_p * rp[(size_t)(s - 1) * P + i];
        const double b = phi_g * rg[(size_t)(s - 1) * P + i];
        for (int d = 0; d < D; ++d) {
          const double xi = x[i * D + d];
          const double vi = omega * v[i * D + d] + a * (pb[i * D + d] - xi) + b * (gb[(size_t)g * D + d] - xi);
          v[i * D + d] = vi;
          x[i * D + d] = xi + vi;
        }
      }
    if ((st = score()) != IQS_OK) return st;
    record(s);
  }
  for (int g = 0; g < G; ++g) {
    best_val[g] = gval[g];
    for (int d = 0; d < D; ++d) best_pos[(size_t)g * D + d] = gb[(size_t)g * D + d];
  }
  return IQS_OK;
}

}  // extern "C"
