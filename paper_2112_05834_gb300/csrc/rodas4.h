// RODAS4 coefficients in the transformed form used by the device stepper.
//
// Hairer & Wanner, Solving ODEs II, Sec. VI.4 (method RODAS, order 4 with an
// embedded order-3 solution, stiffly accurate) written in the variables
// u_i = sum_j gamma_ij k_j of Sec. IV.7 (Eq. 7.3 and the remark after it), so a
// stage needs no Jacobian-vector product:
//   (I/(h gamma) - J) u_i = f(y0 + sum_{j<i} a_ij u_j) + sum_{j<i} (c_ij / h) u_j
//   y1 = y0 + sum_i m_i u_i,   error estimate = sum_i e_i u_i = u_6.
// The method is stiffly accurate, so stage 6 is evaluated at the embedded
// solution and stage 5 and 6 share a_5j; m = (a_51, .., a_54, 1, 1).
#pragma once

namespace chem {

constexpr double kRodasGamma = 0.25;

#define CHEM_RODAS_A                                                                     \
  {                                                                                      \
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0},                                                      \
    {1.544, 0.0, 0.0, 0.0, 0.0, 0.0},                                                    \
    {0.9466785280815826, 0.2557011698983284, 0.0, 0.0, 0.0, 0.0},                        \
    {3.314825187068521, 2.896124015972201, 0.9986419139977817, 0.0, 0.0, 0.0},           \
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.687886036105895, 0.0,   \
     0.0},                                                                               \
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.687886036105895, 1.0,   \
     0.0},                                                                               \
  }
constexpr double kRodasA[6][6] = CHEM_RODAS_A;

#define CHEM_RODAS_C                                                                     \
  {                                                                                      \
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0},                                                      \
    {-5.6688, 0.0, 0.0, 0.0, 0.0, 0.0},                                                  \
    {-2.430093356833875, -0.2063599157091915, 0.0, 0.0, 0.0, 0.0},                       \
    {-0.1073529058151375, -9.594562251023355, -20.47028614809616, 0.0, 0.0, 0.0},        \
    {7.496443313967647, -10.24680431464352, -33.99990352819905, 11.7089089320616, 0.0,   \
     0.0},                                                                               \
    {8.083246795921522, -7.981132988064893, -31.52159432874371, 16.31930543123136,       \
     -6.058818238834054, 0.0},                                                           \
  }
constexpr double kRodasC[6][6] = CHEM_RODAS_C;

#define CHEM_RODAS_M \
  {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.687886036105895, 1.0, 1.0}
constexpr double kRodasM[6] = CHEM_RODAS_M;
constexpr double kRodasE[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.0};

// Step-size control (Hairer & Wanner II, Sec. IV.8): h_new = h * clamp(safety * err^(-1/4)).
constexpr double kSafety = 0.9, kFacMin = 0.2, kFacMax = 5.0, kHmin = 1e-20;

}  // namespace chem
