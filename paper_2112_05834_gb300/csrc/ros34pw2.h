// ROS34PW2 coefficients in the original form (J. Rang and L. Angermann, "New
// Rosenbrock W-methods of order 3 for partial differential algebraic equations of
// index 1", BIT 45 (2005)):
//   (I - h gamma W) k_i = h f(y0 + sum_{j<i} alpha_ij k_j) + h W sum_{j<i} gamma_ij k_j,
//   y1 = y0 + sum b_i k_i, embedded yhat = y0 + sum bhat_i k_i.
// Four stages, order 3 for ANY matrix W (a W-method: the order does not rely on W
// being the exact Jacobian), embedded order 2, stiffly accurate, L-stable. The host
// converts them to the transformed form of the device stepper (see rodas4.h).
#pragma once

namespace chem {

constexpr double kRos34Gamma = 4.3586652150845900e-01;
constexpr double kRos34Alpha[4][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {8.7173304301691801e-01, 0.0, 0.0, 0.0},
    {8.4457060015369423e-01, -1.1299064236484185e-01, 0.0, 0.0},
    {0.0, 0.0, 1.0, 0.0}};
// Gamma below the diagonal (the diagonal is kRos34Gamma)
constexpr double kRos34Gam[4][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {-8.7173304301691801e-01, 0.0, 0.0, 0.0},
    {-9.0338057013044082e-01, 5.4180672388095326e-02, 0.0, 0.0},
    {2.4212380706095346e-01, -1.2232505839045147e+00, 5.4526025533510214e-01, 0.0}};
constexpr double kRos34B[4] = {2.4212380706095346e-01, -1.2232505839045147e+00, 1.5452602553351020e+00,
                               4.3586652150845900e-01};
constexpr double kRos34Bhat[4] = {3.7810903145819369e-01, -9.6042292212423178e-02, 5.0000000000000000e-01,
                                  2.1793326075422950e-01};

}  // namespace chem
