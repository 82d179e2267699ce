// Host-side helpers shared by the translation units that define C entry points
// (defined in sc_api.cu).
#pragma once

#include "sc_profile.cuh"

namespace scgb {

// Record the calling thread's sc_last_error() message and return st.
sc_status set_error(sc_status st, const char *msg);

// Checks of the model part of sc_params that every entry point taking params
// applies: lattice size (>= 1, at most 2^31 - 1 sites), lattice, stencil (E6
// needs D3Q19, D2Q9 needs nz == 1), psi_self and finite couplings.
sc_status validate_model(const sc_params *p);

// Checks of a profile request for a lattice of these params: known kind,
// 1 <= nbins <= max_bins, nbins <= nx for the x-axis line (one site per row),
// bin_width > 0 for radial shells, finite centre.
sc_status validate_profile_request(const sc_params *p, int32_t kind, const double centre[3], double bin_width,
                                   int32_t nbins, int32_t max_bins);

// ProfileArgs of a validated request (chunk set by the launcher).
ProfileArgs profile_args(const sc_params *p, int32_t kind, const double centre[3], double bin_width, int32_t nbins);

}  // namespace scgb
