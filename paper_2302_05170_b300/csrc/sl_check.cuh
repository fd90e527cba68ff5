// sl_check.cuh -- host-side argument checks shared by the online samplers.
#pragma once

#include "../../include/sevenleague.h"

namespace sl {

// Number of parameters theta of an exact-collocation model (2 for GBM, 3 for OU).
int model_p(int model);
// The network descriptor against (m, p): shape, activation, precision, d_in limits.
int check_net(const sl_net* net, int m, int p);
// Model, m, n_steps, T, theta and (for SL_MODEL_MLP) the network.
int check_common(int model, const sl_net* net, const float* theta, int p, float T, int n_steps, int m);

}  // namespace sl
