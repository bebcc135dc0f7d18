/* Prints sizeof / offsetof of the public structs of include/pfarna.h, so the
 * test-suite can check the ctypes mirrors against the C compiler's layout. */
#include <stddef.h>
#include <stdio.h>

#include "pfarna.h"

#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m))

int main(void) {
  printf("pf_track_config sizeof %zu\n", sizeof(pf_track_config));
  F(pf_track_config, G); F(pf_track_config, Np); F(pf_track_config, H); F(pf_track_config, W);
  F(pf_track_config, patch_radius); F(pf_track_config, mode); F(pf_track_config, sigma_psf);
  F(pf_track_config, background); F(pf_track_config, sigma_obs); F(pf_track_config, sigma_pos);
  F(pf_track_config, sigma_v); F(pf_track_config, sigma_I); F(pf_track_config, ex_ratio);
  F(pf_track_config, pe_eff_cutoff); F(pf_track_config, init_kind); F(pf_track_config, init_state);
  F(pf_track_config, init_lo); F(pf_track_config, init_hi); F(pf_track_config, init_radius);
  F(pf_track_config, obs_model); F(pf_track_config, seed); F(pf_track_config, track_id);
  F(pf_track_config, record_ancestors); F(pf_track_config, resample_rule); F(pf_track_config, ess_fraction);
  F(pf_track_config, send_rule); F(pf_track_config, topology); F(pf_track_config, node_groups);
  printf("pf_step_stats sizeof %zu\n", sizeof(pf_step_stats));
  F(pf_step_stats, step); F(pf_step_stats, n_ex); F(pf_step_stats, pe_eff); F(pf_step_stats, log_c);
  F(pf_step_stats, log_Z); F(pf_step_stats, xhat); F(pf_step_stats, degenerate_groups);
  F(pf_step_stats, resampled_groups);
  return 0;
}
