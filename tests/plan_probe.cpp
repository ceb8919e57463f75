// Host-side probe of the collision plan builder (test infrastructure, no GPU needed): reads
// a plan description from stdin, runs dgfs::build_plan (host code only: quadrature rules,
// design, radii, task and entry lists, table slot codes) and prints what it built as one
// JSON object.  tests/test_plan_host.py compiles it against libdgfs.so.
//
// stdin: N L s precision flags N_rho M has_sigma R
//        mass[s]  omega[s*s]  alpha[s*s]  (has_sigma: sigma[3M] w_sigma[M])
#include <cstdio>
#include <vector>

#include "dgfs_internal.h"

int main() {
  dgfs_plan_desc d = {};
  int has_sigma = 0;
  if (std::scanf("%d %lf %d %d %u %d %d %d %lf", &d.N, &d.L, &d.s, &d.precision, &d.flags, &d.N_rho, &d.M,
                 &has_sigma, &d.R) != 9)
    return 2;
  const int s = d.s;
  std::vector<double> mass(s), omega(s * s), alpha(s * s), sigma, w_sigma;
  for (double& v : mass) std::scanf("%lf", &v);
  for (double& v : omega) std::scanf("%lf", &v);
  for (double& v : alpha) std::scanf("%lf", &v);
  if (has_sigma) {
    sigma.resize(3 * d.M);
    w_sigma.resize(d.M);
    for (double& v : sigma) std::scanf("%lf", &v);
    for (double& v : w_sigma) std::scanf("%lf", &v);
    d.sigma = sigma.data();
    d.w_sigma = w_sigma.data();
  }
  d.mass = mass.data();
  d.omega = omega.data();
  d.alpha = alpha.data();
  dgfs::Plan p;
  const int rc = dgfs::build_plan(&d, p);
  std::printf("{\"rc\": %d", rc);
  if (rc == DGFS_OK) {
    std::printf(", \"R\": %.17g, \"vss\": %d, \"antipodal\": %d, \"n_fslot\": %d, \"max_ent\": %d", p.R,
                p.vss ? 1 : 0, p.antipodal ? 1 : 0, p.n_fslot, p.max_ent);
    std::printf(", \"n_t\": %d, \"vss_a_max\": %.17g", p.n_t, p.vss_a_max);
    std::printf(", \"fslot\": [");
    for (size_t k = 0; k < p.fslot.size(); ++k) std::printf("%s%d", k ? ", " : "", p.fslot[k]);
    std::printf("], \"sigma\": [");
    for (size_t k = 0; k < p.sigma.size(); ++k) std::printf("%s%.17g", k ? ", " : "", p.sigma[k]);
    std::printf("], \"w_sigma\": [");
    for (size_t k = 0; k < p.w_sigma.size(); ++k) std::printf("%s%.17g", k ? ", " : "", p.w_sigma[k]);
    std::printf("], \"tasks\": [");
    for (size_t t = 0; t < p.tasks.size(); ++t) {
      const dgfs::TaskDesc& tk = p.tasks[t];
      std::printf("%s{\"i\": %d, \"j\": %d, \"out0\": %d, \"out1\": %d, \"groups\": [", t ? ", " : "", tk.i, tk.j,
                  tk.out0, tk.out1);
      for (int g = 0; g < tk.n_grp; ++g) {
        const dgfs::GroupDesc& gd = p.groups[tk.grp_off + g];
        std::printf("%s[%d, %d]", g ? ", " : "", gd.first, gd.count);
      }
      std::printf("], \"entries\": [");
      for (int e = 0; e < tk.n_ent; ++e) {
        const int k = tk.ent_off + e;
        std::printf("%s{\"m\": %d, \"w\": %.17g, \"code0\": %d, \"code1\": %d, \"ysh\": %d}", e ? ", " : "",
                    p.ent_sigma[k], p.ent_w[k], p.ent_m[2 * k], p.ent_m[2 * k + 1], p.ent_ysh[k]);
      }
      std::printf("]}");
    }
    std::printf("], \"pair_R\": [");
    for (size_t k = 0; k < p.pair_R.size(); ++k) std::printf("%s%.17g", k ? ", " : "", p.pair_R[k]);
    std::printf("]");
  }
  std::printf("}\n");
  return 0;
}
