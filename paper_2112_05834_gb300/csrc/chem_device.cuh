// Device code of the batched stiff-chemistry integrator (sm_103a), shared by the
// translation units that instantiate the integration kernel (chem_kernels.cu: the
// RODAS4 stepper, diagnostics and launchers; chem_kernels_w.cu: the W-method).
//
// One CTA integrates one cell at a time; its warps share the cell's work:
// species and 32-reaction chunks are dealt over threads and warps for the rates,
// Jacobian rows over warps (columns over lanes) for the assembly; the FP64 form
// factorises in shared memory (rows over warps) and solves on one warp, the mixed
// form inverts in FP32 with the matrix in registers (columns over warps, rows over
// lanes) and solves by matrix-vector products over all threads. All per-cell data
// (state, stage vectors, per-reaction derivative data, the iteration matrix) lives
// in shared memory, except that the mixed form may keep its assembled matrix (float-
// float pairs) in a global-memory slot of the CTA when that lets more CTAs share an SM; the
// mechanism tables are read through the L1 cache.
//
// Paper mapping: rates and RHS = pyJac's reaction-rate evaluation; analytic
// Jacobian = pyJac's Jacobian (Methodology, "Analytical Jacobian and improved ODE
// solution"); LU + substitution = the LAPACK replacement of OpenFOAM's linear
// algebra (same section); the per-cell loop = the implicit ODE solver of the
// Introduction; the work queue = DLBFoam's redistribution of cell problems
// (Methodology, "DLBFoam: Dynamic load balancing"), reinterpreted inside one GPU.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "chem.h"
#include "chem_internal.h"
#include "chem_kernels.h"
#include "rodas4.h"

namespace chem {

#define FULLMASK 0xffffffffu

// ---------------------------------------------------------------------------
// Float-float arithmetic (a value is hi + lo with two FP32 numbers, |lo| below ulp(hi)):
// error-free products with FMA (Dekker's TwoProduct) and sums by Knuth's TwoSum
// give about 44-48 significant bits on the FP32 pipe. On GB300 an SM's FP32 pipe
// completes 64 times the operations per clock of its FP64 pipe, which the
// integration keeps busy, so the mixed form runs its long sums of products here:
// third-body concentrations, the Jacobian assembly and the refinement residuals.
// The _rn intrinsics keep the compiler from contracting a product and a sum into
// one FMA, which would break the error-free transformations.
// ---------------------------------------------------------------------------
struct __align__(8) ff2 {
  float hi, lo;
};
// Conversions between FP64 and FP32 run on the FP64 pipe on this part, at its rate,
// so the splits and widenings below use integer operations on the bit patterns.
// Double to float-float: hi = x truncated to 24 significant bits, lo = x - hi (the
// 29 remaining mantissa bits, rounded to 24 by the integer-to-float conversion and
// scaled by an exact power of two). In FP32's subnormal range (2^-149 <= |x| <
// 2^-126) hi = x truncated to a multiple of 2^-149 and lo = 0; below it (0, 0);
// |x| >= 2^128 gives +-inf (NaN stays NaN) with lo = 0.
__device__ __forceinline__ ff2 ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const float m = __uint2float_rn(lw & 0x1FFFFFFFu);
  // m 2^(e - 1075) as one power-of-two factor for e >= 949, else as 2^(e - 1011) 2^-64
  const bool big = e >= 949;
  const float s1 = __uint_as_float((unsigned)(big ? e - 948 : e - 884) << 23);
  const float s2 = big ? 1.0f : __uint_as_float(0x1F800000u);  // 2^-64
  ff2 r = {__uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29)),
           __uint_as_float(__float_as_uint(__fmul_rn(__fmul_rn(m, s1), s2)) | sgn)};
  if (e < 897) {
    const int sh = 926 - e;  // the 53-bit significand times 2^(e - 1075) in units of 2^-149
    const unsigned frac = sh <= 52 ? (unsigned)(((1ull << 52) | (b & 0xFFFFFFFFFFFFFull)) >> sh) : 0u;
    r = {__uint_as_float(sgn | frac), 0.0f};
  }
  if (e > 1150) {
    const bool nan = e == 2047 && ((hw & 0xFFFFFu) | lw) != 0u;
    r = {__uint_as_float(sgn | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.0f};
  }
  return r;
}
// float to double, exactly
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu, mant = u & 0x7FFFFFu, sgn = u & 0x80000000u;
  unsigned hw = sgn | ((e + 896u) << 20) | (mant >> 3), lw = mant << 29;
  if (e == 0u) {
    // zero or subnormal mant 2^-149 = 2^(p - 149) (1 + f), p = position of the leading bit
    const int p = 31 - __clz(mant);
    const unsigned long long fr = (unsigned long long)mant << (52 - p);
    hw = mant ? sgn | ((unsigned)(p + 874) << 20) | ((unsigned)(fr >> 32) & 0xFFFFFu) : sgn;
    lw = mant ? (unsigned)fr : 0u;
  } else if (e == 255u) {
    hw = sgn | 0x7FF00000u | (mant >> 3) | (mant ? 0x80000u : 0u);
    lw = 0u;
  }
  return __hiloint2double((int)hw, (int)lw);
}
__device__ __forceinline__ double ff_value(ff2 a) { return f32_to_f64(a.hi) + f32_to_f64(a.lo); }
__device__ __forceinline__ ff2 ff_neg(ff2 a) { return {-a.hi, -a.lo}; }
// s + e renormalised, |s| >= |e| (or s == 0)
__device__ __forceinline__ ff2 fast_two_sum(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
// a + b = s + e exactly (Knuth)
__device__ __forceinline__ ff2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
  const ff2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff2 ff_sub(ff2 a, ff2 b) { return ff_add(a, ff_neg(b)); }
// hi * hi exactly, plus the cross terms (the lo * lo term is below the precision kept)
__device__ __forceinline__ ff2 ff_prod(ff2 a, ff2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return {p, e};  // not renormalised
}
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
  const ff2 p = ff_prod(a, b);
  return fast_two_sum(p.hi, p.lo);
}
// a * b + c
__device__ __forceinline__ ff2 ff_fma(ff2 a, ff2 b, ff2 c) {
  const ff2 p = ff_prod(a, b);
  const ff2 s = two_sum(p.hi, c.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(p.lo, c.lo)));
}
// Running float-float sum s + c in the manner of Ogita, Rump and Oishi's Sum2/Dot2:
// each term's hi part enters s through TwoSum, its rounding error, its lo part and the
// cross terms of a product gather in c; renormalised once at the end. Each term waits
// on one FP32 add of the previous one (s and c are separate chains), where a chain of
// renormalised float-float sums waits on about eight.
struct ff_sum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ ff_sum() = default;
  __device__ __forceinline__ explicit ff_sum(ff2 v) : s(v.hi), c(v.lo) {}
  __device__ __forceinline__ void add(ff2 v) {
    const ff2 t = two_sum(s, v.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, v.lo));
  }
  __device__ __forceinline__ void add_prod(ff2 a, ff2 b) {
    const ff2 p = ff_prod(a, b);
    const ff2 t = two_sum(s, p.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, p.lo));
  }
  __device__ __forceinline__ ff2 value() const { return fast_two_sum(s, c); }
};

// conversions between the matrix element types (double, float, float-float)
__device__ __forceinline__ float to_float(float a) { return a; }
__device__ __forceinline__ float to_float(double a) { return (float)a; }
__device__ __forceinline__ float to_float(ff2 a) { return a.hi; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(ff2 a) { return ff_value(a); }
template <class R>
__device__ __forceinline__ R from_double(double a) {
  if constexpr (std::is_same<R, ff2>::value) return ff_split(a);
  else return (R)a;
}

// ---------------------------------------------------------------------------
// Exponential by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15(2), 1989), with a 256-entry table: x = (256 m + j) ln2/256 + r with
// |r| <= ln2/512, so exp(x) = 2^m 2^(j/256) exp(r). 2^(j/256) comes from a table of
// (lead, trail) pairs (lead = 2^(j/256) rounded to double, trail = the remainder
// rounded to double), exp(r) - 1 from its Taylor polynomial of degree 4 (truncation
// r^5/120 < 3.8e-17 relative), ln2/256 as a two-term split for the reduction, and
// 2^m is added to the exponent field. |x| >= 672, infinities and NaN take the
// library exp. Ten FP64 instructions; the table (4 KB) is read through the L1 cache.
// ---------------------------------------------------------------------------
static __device__ const double2 g_exp2_tab[256] = {
    {1.0, 0.0},
    {1.0027112750502025, -3.636615928692264e-17},
    {1.0054299011128027, 9.499186535455032e-17},
    {1.0081558981184175, -3.252058756084308e-17},
    {1.0108892860517005, -1.5234778603368577e-17},
    {1.0136300849514894, 9.283599768183568e-18},
    {1.016378314910953, -5.77217007319966e-17},
    {1.019133996077738, 3.601904982259662e-17},
    {1.0218971486541166, 5.109225028973444e-17},
    {1.0246677928971357, -7.56160786848778e-17},
    {1.0274459491187637, -4.9560741746453704e-17},
    {1.030231637686041, 3.319830041080813e-17},
    {1.0330248790212284, 7.600838874027088e-18},
    {1.0358256936019572, -7.806782391337636e-17},
    {1.0386341019613787, 5.996273788852511e-17},
    {1.041450124688316, 3.784830480287576e-17},
    {1.0442737824274138, 8.551889705537965e-17},
    {1.0471050958792898, 7.277077243104315e-17},
    {1.0499440858006872, 5.592937848127003e-17},
    {1.0527907730046264, -9.629482899026936e-17},
    {1.0556451783605572, 1.759325738772092e-18},
    {1.0585073227945128, -7.152651856637781e-17},
    {1.061377227289262, -1.1973537085365658e-17},
    {1.0642549128844645, 5.0787541986112304e-17},
    {1.0671404006768237, -7.899853966841582e-17},
    {1.0700337118202419, -9.937162711288919e-17},
    {1.0729348675259756, -3.839668843358824e-18},
    {1.075843889062791, -1.0002716151144136e-17},
    {1.0787607977571199, -6.656660436056593e-17},
    {1.0816856149932152, -4.782623902997086e-17},
    {1.0846183622133092, 3.166152845816346e-17},
    {1.0875590609177697, 5.409349307820291e-18},
    {1.0905077326652577, -3.046782079812471e-17},
    {1.0934643990728858, 1.441395814726921e-17},
    {1.0964290818163769, -5.919933484449316e-17},
    {1.099401802630222, 7.170459599701923e-17},
    {1.102382583307841, 5.2660368715706944e-17},
    {1.1053714457017412, 8.239288760500214e-17},
    {1.1083684117236787, -8.786813845180527e-17},
    {1.1113735033448175, 5.563945026669698e-17},
    {1.1143867425958924, 1.0410278456845571e-16},
    {1.1174081515673693, -7.97680590262822e-17},
    {1.1204377524096067, -6.201085906554179e-17},
    {1.12347556733302, -9.699737588987043e-17},
    {1.1265216186082418, 5.165856758795457e-17},
    {1.129575928566288, 6.712805858726257e-17},
    {1.1326385195987192, 3.237356166738e-17},
    {1.1357094141578055, 5.066599926126156e-17},
    {1.1387886347566916, 8.912812676025408e-17},
    {1.1418762039695616, 4.6510911775314124e-17},
    {1.1449721444318042, 4.6412898921700107e-17},
    {1.148076478840179, 6.897740236627192e-17},
    {1.1511892299529827, 3.250710218863827e-17},
    {1.154310420590216, 1.0417128946273266e-16},
    {1.1574400736337511, -9.1238712311344e-17},
    {1.1605782120274988, -3.261040205417394e-17},
    {1.1637248587775775, 3.8292048369240935e-17},
    {1.1668800369524817, -8.79187957999917e-17},
    {1.1700437696832502, -1.8477442017900047e-18},
    {1.1732160801636373, -7.287562586584994e-17},
    {1.1763969916502812, 5.554203254218079e-17},
    {1.1795865274628758, 1.009231277510039e-16},
    {1.182784710984341, 1.542975430079076e-17},
    {1.1859915656609938, -9.209506835293106e-18},
    {1.189207115002721, 3.982015231465646e-17},
    {1.1924313825831512, 4.3975514156097214e-17},
    {1.1956643920398273, 4.6166036704814814e-17},
    {1.1989061670743806, -9.809193356008423e-17},
    {1.202156731452703, 6.644981499252301e-17},
    {1.2054161090051239, -3.3572721932675296e-17},
    {1.2086843236265816, -4.746725945228984e-17},
    {1.2119613992768012, -4.8906110775211184e-17},
    {1.215247359980469, -7.712630692681488e-17},
    {1.2185422298274085, -9.006726958363838e-17},
    {1.2218460329727576, -1.0611021211402691e-16},
    {1.2251587936371455, -8.903533814269983e-17},
    {1.22848053610687, -1.89878163130253e-17},
    {1.2318112847340759, 7.38938247161005e-17},
    {1.2351510639369334, -1.0755244344307841e-16},
    {1.2384998981998165, 2.7677020555739674e-17},
    {1.241857812073484, 4.658027591836937e-17},
    {1.245224830175258, -4.6772404498467275e-17},
    {1.2486009771892048, -8.261810999021964e-17},
    {1.2519862778663162, 4.8341671524698976e-17},
    {1.255380757024691, -6.7113898212968784e-18},
    {1.2587844395497165, -8.421782587730599e-17},
    {1.2621973503942507, -3.0844648874738465e-17},
    {1.2656195145788063, 4.2505770034508686e-17},
    {1.2690509571917332, 2.667932131342186e-18},
    {1.2724917033894028, -1.0577916267212421e-17},
    {1.275941778396392, 9.91543024421429e-17},
    {1.2794012075056693, -9.759095008356062e-17},
    {1.2828700160787783, 1.713594918243561e-17},
    {1.2863482295460256, -3.416955706936182e-17},
    {1.2898358734066657, 8.949257530897592e-17},
    {1.2933329732290895, -2.9745904431327516e-17},
    {1.2968395546510096, 2.5382502794888315e-17},
    {1.3003556433796506, 5.678728102802217e-17},
    {1.3038812651919358, 8.647675598267871e-17},
    {1.3074164459346773, -7.336645652878869e-17},
    {1.3109612115247644, -7.181536135519454e-17},
    {1.3145155879493546, 2.2675433151045856e-17},
    {1.318079601266064, -5.4579558271491535e-17},
    {1.3216532776031575, -2.4806382459130217e-17},
    {1.3252366431597413, -2.8587312100388614e-17},
    {1.3288297242059544, 4.08908622391016e-17},
    {1.3324325470831615, -5.101586630916744e-17},
    {1.3360451382041458, -5.891866356388801e-17},
    {1.339667524053303, 8.927282594831732e-17},
    {1.3432997311868353, -5.802580890201438e-17},
    {1.3469417862329458, 3.224065101254679e-17},
    {1.3505937158920345, -8.287110381462417e-17},
    {1.3542555469368927, 7.70094837980299e-17},
    {1.3579273062129011, -9.529635744825189e-17},
    {1.3616090206382248, 1.533787661270668e-18},
    {1.365300717204012, -1.0005363125974765e-16},
    {1.3690024229745905, 9.593797919118849e-17},
    {1.3727141650876684, -4.495960595234841e-17},
    {1.3764359707545302, -6.898588935871801e-17},
    {1.380167867260238, 1.0510314579969984e-16},
    {1.383909881963832, -6.770511658794786e-17},
    {1.387662042298529, 8.422984274875415e-17},
    {1.3914243757719262, -4.9061748652889893e-17},
    {1.3951969099662003, -9.329336224225497e-17},
    {1.3989796725383112, -9.614213209051323e-17},
    {1.4027726912202048, -5.295783249407989e-17},
    {1.4065759938190154, 7.034914812136422e-18},
    {1.4103896082172707, 4.166548728435062e-17},
    {1.4142135623730951, -9.667293313452913e-17},
    {1.4180478843204152, 2.2744385421855295e-17},
    {1.4218926021691656, -1.6077828915890244e-17},
    {1.4257477441054942, 9.880690758500607e-17},
    {1.42961333839197, -1.2031642489053655e-17},
    {1.433489413367789, -5.802454243926826e-17},
    {1.4373759974489824, -4.2040340164675566e-17},
    {1.4412731191286257, 5.602503650878986e-18},
    {1.4451808069770467, -3.0237581349939873e-17},
    {1.449099089642035, -6.259405000819309e-17},
    {1.4530279958490526, -5.779948609396106e-17},
    {1.4569675544014438, 5.648679453876998e-17},
    {1.460917794180647, -5.600377186075216e-17},
    {1.4648787441464057, 9.530767543587157e-17},
    {1.4688504333369818, 8.465882756533628e-17},
    {1.4728328908693675, 6.691774081940589e-17},
    {1.4768261459394993, -3.483994556892796e-17},
    {1.4808302278224719, -9.686952102630619e-17},
    {1.4848451658727524, 1.0780086764407481e-16},
    {1.488870989524397, 6.155367157742871e-17},
    {1.4929077282912648, 1.4192920154284036e-17},
    {1.4969554117672355, -2.861663253899158e-17},
    {1.5010140696264256, -6.413767275790235e-17},
    {1.5050837316234065, 7.074710613582846e-17},
    {1.5091644275934228, -1.016455327754295e-16},
    {1.5132561874526098, 8.884497851338712e-17},
    {1.5173590411982147, -4.308699472043341e-17},
    {1.5214730189088146, -5.9963876759456834e-18},
    {1.5255981507445384, -1.1024941712342561e-16},
    {1.529734466947287, 3.7857921151572197e-17},
    {1.533881997840956, 8.875226844438446e-17},
    {1.5380407738316568, 1.0174672351161359e-16},
    {1.5422108254079407, 7.949834809697621e-17},
    {1.5463921831410214, 1.068396000565722e-16},
    {1.550584877685, -1.4600706590689385e-17},
    {1.5547889397770887, -8.003161350116036e-17},
    {1.559004400237837, 3.7812070533575275e-17},
    {1.5632312899713576, 7.484777645590734e-17},
    {1.567469639965553, -1.0352061768849722e-16},
    {1.5717194812923414, -3.3429840046872e-17},
    {1.5759808451078865, -1.0136916471278304e-17},
    {1.5802537626528246, -5.163402929554468e-17},
    {1.5845382652524937, -1.9337717034585703e-17},
    {1.588834384317164, -5.9949501188244794e-18},
    {1.593142151342267, -1.0094406542311964e-16},
    {1.597461597908627, 2.4868392796221e-17},
    {1.6017927556826934, -6.054917453527784e-17},
    {1.606135656416771, -1.0354545288059995e-16},
    {1.6104903319492543, 2.4707192569797888e-17},
    {1.6148568142048607, -7.316663399125123e-17},
    {1.6192351351948637, 2.0941334154229092e-17},
    {1.6236253270173289, -3.584512851414475e-17},
    {1.6280274218573478, -6.712955084707084e-17},
    {1.632441451987275, 9.852819230429993e-17},
    {1.6368674497669644, 7.698325071319876e-17},
    {1.6413054476440063, -9.247568737640706e-17},
    {1.645755478153965, -1.0125679913674773e-16},
    {1.6502175739206177, 9.133279588729904e-18},
    {1.6546917676561943, 9.643294303196029e-17},
    {1.6591780921616162, -7.275545550823051e-17},
    {1.6636765803267364, 5.8909926967131e-17},
    {1.6681872651305825, 4.269178019570615e-17},
    {1.6727101796415966, -5.476715964599563e-17},
    {1.6772453570178785, 8.303949509950733e-17},
    {1.681792830507429, 8.199010020581497e-17},
    {1.6863526334483934, -7.181463278358011e-17},
    {1.6909247992693053, -9.66967147439488e-17},
    {1.6955093614893326, 7.238416872845167e-17},
    {1.7001063537185235, -8.0237193703977e-18},
    {1.7047158096580513, -2.7288832847972816e-17},
    {1.709337763100463, -9.868779456632931e-17},
    {1.713972247929926, 6.473975107753367e-17},
    {1.718619298122478, -1.851380418263111e-17},
    {1.723278947746274, -9.5221238003938e-17},
    {1.7279512309618377, -1.0750981861204642e-16},
    {1.732636182022311, -1.6980510743154155e-18},
    {1.7373338352737062, 3.164389299292957e-17},
    {1.7420442251551564, -1.5259591189507888e-18},
    {1.746767386199169, -1.0752290483507515e-16},
    {1.7515033530318782, -5.1244504205967247e-17},
    {1.7562521603732995, 2.960140695448873e-17},
    {1.761013843037584, -7.943253125039228e-17},
    {1.7657884359332727, 9.461315018083268e-17},
    {1.7705759740635547, 5.961794510040556e-17},
    {1.7753764925265212, 6.429731796556572e-17},
    {1.7801900265154245, -5.2846272890916174e-17},
    {1.785016611318935, 1.5330400121031314e-17},
    {1.789856282321401, -4.1543546606833504e-17},
    {1.7947090750031072, 1.8227458427912087e-17},
    {1.7995750249405351, -2.526889233358898e-17},
    {1.804454167806624, -5.177222408793318e-17},
    {1.809346539371032, -9.03264140245003e-17},
    {1.8142521755003989, -9.969531538920349e-17},
    {1.8191711121586085, 7.402676901145839e-17},
    {1.8241033854070534, -1.0159627862277083e-16},
    {1.8290490314048973, 6.889192908835696e-17},
    {1.8340080864093424, 3.283107224245627e-17},
    {1.8389805867758937, 6.918969740272512e-18},
    {1.843966568958626, -5.939742026949965e-17},
    {1.8489660695104508, 9.027580446261089e-17},
    {1.8539791250833855, 9.761887490727594e-17},
    {1.8590057724288205, -9.528705461989941e-17},
    {1.864046048397789, 6.540912680620572e-17},
    {1.8690999899412386, -9.938505214255067e-17},
    {1.8741676341103, -6.122763413004143e-17},
    {1.8792490180565602, -1.6226315557835845e-17},
    {1.8843441790323345, -8.226593125533711e-17},
    {1.8894531543909392, -9.005168285059127e-17},
    {1.8945759815869656, 3.4034035352165297e-17},
    {1.8997126981765553, -3.8597397693785143e-17},
    {1.9048633418176741, 6.533857514718279e-17},
    {1.9100279502703899, -5.90968800674406e-17},
    {1.9152065613971474, -1.0619946056195963e-16},
    {1.9203992131630474, 7.116681540630314e-17},
    {1.925605943636125, -9.914963769693741e-17},
    {1.930826790987627, 6.16714970616911e-17},
    {1.9360617934922943, 1.0332385960676326e-16},
    {1.9413109895286405, -6.638029891621488e-17},
    {1.9465744175792332, 6.811022349533877e-17},
    {1.9518521162309783, -2.199016969979351e-17},
    {1.9571441241754002, 8.960767791036668e-17},
    {1.9624504802089273, 1.0976844000913547e-16},
    {1.9677712232331759, -1.0314928011531132e-16},
    {1.9731063922552343, -7.451617863956037e-18},
    {1.978456026387951, 4.0388753109278167e-17},
    {1.9838201648502194, -2.2034544123910627e-17},
    {1.9891988469672663, 8.2051326383692e-18},
    {1.9945921121709402, 1.7909710352002645e-17},
};

static __device__ __noinline__ double exp_outside(double x) { return exp(x); }

constexpr double kInvLn10 = 0.43429448190325176;  // 1 / ln 10
constexpr double kLnRcP0 = 4.407418589020958;  // ln(Rc / P0), cgs

__device__ __forceinline__ double xexp(double x) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40850000) return exp_outside(x);  // |x| >= 672, inf, NaN
  constexpr double kInvL = 369.3299304675746;      // 256 / ln 2
  constexpr double kL1 = 0.0027076061740622863;    // ln2/256 rounded to double
  constexpr double kL2 = 9.058776616587108e-20;    // ln2/256 - kL1
  constexpr double kShift = 6755399441055744.0;    // 1.5 * 2^52: rounds to an integer in the low word
  const double t = fma(x, kInvL, kShift);
  const int N = __double2loint(t);
  const double2 sj = __ldg(&g_exp2_tab[N & 255]);
  const double Nd = t - kShift;
  double r = fma(-Nd, kL1, x);
  r = fma(-Nd, kL2, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double em1 = fma(r * r, q, r);  // exp(r) - 1
  const double y = sj.x + fma(sj.x, em1, sj.y);
  return __hiloint2double(__double2hiint(y) + (N >> 8) * (1 << 20), __double2loint(y));
}

// ---------------------------------------------------------------------------
// Natural logarithm, table-driven in the manner of Tang (P. T. P. Tang, "Table-
// driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990): x = 2^m y with y in [1, 2), F = 1 + j/128 the
// nearest of 129 points, c = 1/F rounded to double, r = y c - 1 (one FMA rounding,
// |r| <= 1/256 + 2^-30), and ln x = m ln 2 - ln c + ln(1 + r), with ln(1 + r) from
// its Taylor series to degree 7 (truncation below 2e-18 relative). The table holds
// (c, -ln c as lead + trail) for the rounded c; ln 2 is split so m ln2_hi is exact.
// Zero, negative, subnormal, infinite and NaN arguments take the library log.
// ---------------------------------------------------------------------------
static __device__ const double g_log_tab[129][3] = {
    {1.0, 0.0, 0.0},
    {0.9922480620155039, 0.007782140442054963, -1.2819179123343749e-20},
    {0.9846153846153847, 0.015504186535965199, -3.2783210228924137e-19},
    {0.9770992366412213, 0.023167059281534418, -3.095927552179262e-19},
    {0.9696969696969697, 0.03077165866675366, 1.0431732029005972e-18},
    {0.9624060150375939, 0.03831886430213666, -2.3579961573512846e-18},
    {0.9552238805970149, 0.04580953603129422, 1.6823639049745016e-19},
    {0.9481481481481482, 0.05324451451881224, 1.803871134979952e-18},
    {0.9411764705882353, 0.060624621816434854, 2.6424025938726934e-18},
    {0.9343065693430657, 0.06795066190850778, 3.9239563038692484e-18},
    {0.927536231884058, 0.07522342123758752, -4.195880720316434e-18},
    {0.920863309352518, 0.08244366921107454, -4.707903082046854e-18},
    {0.9142857142857143, 0.08961215868968717, -1.9573659817110993e-18},
    {0.9078014184397163, 0.09672962645855114, -4.0291867005826106e-18},
    {0.9014084507042254, 0.10379679368164355, -3.195893222617445e-18},
    {0.8951048951048951, 0.11081436634029011, 2.0511100808140527e-18},
    {0.8888888888888888, 0.11778303565638351, -1.1971685747593662e-18},
    {0.8827586206896552, 0.12470347850095725, -4.6522609636496624e-18},
    {0.8767123287671232, 0.13157635778871932, 1.112300087972959e-17},
    {0.8707482993197279, 0.1384023228591192, -1.3766819196398948e-17},
    {0.8648648648648649, 0.14518200984449783, 8.242418783022477e-18},
    {0.8590604026845637, 0.151916042025842, 4.1233095848339465e-19},
    {0.8533333333333334, 0.15860503017663852, 2.583386492298558e-18},
    {0.847682119205298, 0.16524957289530717, -9.227573884334224e-18},
    {0.8421052631578947, 0.17185025692665928, -6.022453821011369e-18},
    {0.8366013071895425, 0.17840765747281825, 1.2720936612962572e-17},
    {0.8311688311688312, 0.18492233849401193, -7.384679440503435e-18},
    {0.8258064516129032, 0.19139485299962947, -1.126213516780448e-17},
    {0.8205128205128205, 0.19782574332991992, -7.995487338741543e-18},
    {0.8152866242038217, 0.20421554142869083, 7.9379985298027e-18},
    {0.810126582278481, 0.21056476910734964, 1.136310596906137e-17},
    {0.8050314465408805, 0.2168739383006143, 6.285749669211092e-18},
    {0.8, 0.2231435513142097, -9.091270597324798e-18},
    {0.7950310559006211, 0.2293741010648459, -5.684839459813236e-18},
    {0.7901234567901234, 0.23556607131276697, -2.394337149518734e-18},
    {0.7852760736196319, 0.24171993688714513, 1.323779871210866e-17},
    {0.7804878048780488, 0.2478361639045812, 8.384472133019162e-18},
    {0.7757575757575758, 0.25391520998096345, -7.180735656435798e-18},
    {0.7710843373493976, 0.259957524436926, 2.4167516341742964e-17},
    {0.7664670658682635, 0.2659635484971379, 1.35209848201012e-19},
    {0.7619047619047619, 0.2719337154836418, 7.833196376974436e-19},
    {0.757396449704142, 0.2778684510034563, 2.2502748630777633e-17},
    {0.7529411764705882, 0.2837681731306446, -6.448868003452105e-18},
    {0.7485380116959064, 0.2896332925830427, 2.0535953219858177e-17},
    {0.7441860465116279, 0.2954642128938359, -7.768320796245443e-18},
    {0.7398843930635838, 0.30126133057816185, -1.5120043309967385e-17},
    {0.735632183908046, 0.3070250352949119, 1.5578716077124932e-18},
    {0.7314285714285714, 0.3127557100038969, -1.3650721793001109e-17},
    {0.7272727272727273, 0.3184537311185346, -6.407962483026777e-19},
    {0.7231638418079096, 0.324119468654212, -4.488767429940198e-18},
    {0.7191011235955056, 0.32975328637246804, -2.5633554999431966e-17},
    {0.7150837988826816, 0.3353555419211378, -1.3746739934976202e-17},
    {0.7111111111111111, 0.3409265869705932, -2.069678002794501e-17},
    {0.7071823204419889, 0.3464667673462086, -3.591951952851805e-18},
    {0.7032967032967034, 0.3519764231571781, 2.0005853013367377e-17},
    {0.6994535519125683, 0.3574558889218038, -2.4269548334425144e-17},
    {0.6956521739130435, 0.3629054936893685, 6.2632141603179415e-18},
    {0.6918918918918919, 0.36832556115870757, 2.690672380132659e-17},
    {0.6881720430107527, 0.373716409793584, -2.449917382477111e-18},
    {0.6844919786096256, 0.3790783529349695, 1.8481479367349684e-17},
    {0.6808510638297872, 0.38441169891033206, 8.164631656028572e-18},
    {0.6772486772486772, 0.38971675114002524, 2.734172667856699e-17},
    {0.6736842105263158, 0.394993808240869, 7.437680769362324e-18},
    {0.6701570680628273, 0.40024316412701266, -1.655340963311913e-17},
    {0.6666666666666666, 0.40546510810816444, -2.881138025962641e-18},
    {0.6632124352331606, 0.4106599249852683, 2.7752739097728695e-17},
    {0.6597938144329897, 0.415827895143711, -5.793440801214822e-18},
    {0.6564102564102564, 0.42096929464412963, 4.5972855136437464e-18},
    {0.6530612244897959, 0.42608439531090014, -7.056391017993593e-19},
    {0.649746192893401, 0.43117346481837143, -1.3539234990021841e-17},
    {0.6464646464646465, 0.43623676677491796, 2.4182887316590065e-17},
    {0.6432160804020101, 0.4412745608048752, 1.0343758877897315e-17},
    {0.64, 0.4462871026284195, 1.6511928324886544e-17},
    {0.6368159203980099, 0.4512746441394586, -9.65179553937242e-18},
    {0.6336633663366337, 0.4562374334815876, 9.07916350878553e-18},
    {0.6305418719211823, 0.46117571512217015, 6.140445034134513e-18},
    {0.6274509803921569, 0.46608972992459924, -2.387354320899491e-19},
    {0.624390243902439, 0.470979715218791, 7.099457177589995e-18},
    {0.6213592233009708, 0.475845904869964, 2.5043069845040313e-17},
    {0.6183574879227053, 0.48068852934575196, -2.7402100563370574e-18},
    {0.6153846153846154, 0.48550781578170077, -1.6618350693852045e-17},
    {0.6124401913875598, 0.4903039880451939, 4.612452524535198e-18},
    {0.6095238095238096, 0.4950772667978514, 1.2508730752094332e-17},
    {0.6066350710900474, 0.49982786955644926, -2.25665388836583e-18},
    {0.6037735849056604, 0.5045560107523953, 1.3275397597891851e-17},
    {0.6009389671361502, 0.5092619017898079, 2.1678544367048826e-17},
    {0.5981308411214953, 0.5139457511022344, -2.4537074021915265e-18},
    {0.5953488372093023, 0.5186077642080457, -1.6859591393570242e-17},
    {0.5925925925925926, 0.5232481437645479, 2.3677269014906905e-17},
    {0.5898617511520737, 0.5278670896208424, -3.071514383985515e-18},
    {0.5871559633027523, 0.5324647988694717, 5.4596227307139745e-17},
    {0.5844748858447488, 0.5370414658968837, -1.9513712761861967e-17},
    {0.5818181818181818, 0.5415972824327444, 1.108461486609421e-17},
    {0.579185520361991, 0.5461324375981356, -6.169692458083718e-18},
    {0.5765765765765766, 0.5506471179526623, -1.3720677478685045e-17},
    {0.5739910313901345, 0.5551415075405016, -1.449278054403172e-17},
    {0.5714285714285714, 0.5596157879354228, -2.8656225429134744e-17},
    {0.5688888888888889, 0.564070138284803, -4.6267923647049475e-17},
    {0.5663716814159292, 0.5685047353526688, -4.0389558221668317e-17},
    {0.5638766519823789, 0.5729197535617854, 4.4242614369063874e-17},
    {0.5614035087719298, 0.5773153650348236, 4.660755938428382e-17},
    {0.5589519650655022, 0.5816917396346225, 2.7912851075301e-17},
    {0.5565217391304348, 0.5860490450035782, -4.272669638447342e-17},
    {0.5541125541125541, 0.5903874466021763, 2.876546074301208e-17},
    {0.5517241379310345, 0.5947071077466928, 2.7629477772138132e-17},
    {0.5493562231759657, 0.5990081896460834, 2.5162534548420983e-17},
    {0.5470085470085471, 0.6032908514380841, 2.0348397202878346e-17},
    {0.5446808510638298, 0.6075552502245418, -4.1692640626751196e-17},
    {0.5423728813559322, 0.6118015411059929, -3.392831249677239e-17},
    {0.540084388185654, 0.616029877215514, 4.9247969628553695e-17},
    {0.5378151260504201, 0.6202404097518576, 3.4764762563436685e-18},
    {0.5355648535564853, 0.6244332880118936, 1.4444646832738594e-17},
    {0.5333333333333333, 0.6286086594223742, -5.360577204673081e-17},
    {0.5311203319502075, 0.6327666695710378, 5.223564575344447e-17},
    {0.5289256198347108, 0.6369074622370692, 2.6473983119023558e-17},
    {0.5267489711934157, 0.6410311794209312, -3.4765774267087093e-17},
    {0.5245901639344263, 0.6451379613735847, -5.110700818729212e-17},
    {0.5224489795918368, 0.6492279466251097, -1.3266356651077771e-17},
    {0.5203252032520326, 0.6533012720127456, -3.7864752792363655e-17},
    {0.5182186234817814, 0.65735807270836, 2.2462005860533567e-17},
    {0.5161290322580645, 0.661398482245365, 2.015224182999491e-17},
    {0.5140562248995983, 0.6654226325450905, 5.424612435933966e-17},
    {0.512, 0.6694306539426292, 7.420657727561746e-18},
    {0.5099601593625498, 0.6734226752121667, 3.84128539325942e-17},
    {0.5079365079365079, 0.6773988235918061, 5.341333284299263e-17},
    {0.5059288537549407, 0.6813592248079031, 1.7765482243852914e-17},
    {0.5039370078740157, 0.6853040030989195, -4.8209665191998585e-17},
    {0.5019607843137255, 0.689233281238809, -9.330006029414747e-18},
    {0.5, 0.6931471805599453, 2.3190468138462996e-17}
};

static __device__ __noinline__ double log_outside(double x) { return log(x); }

__device__ __forceinline__ double xlog(double x) {
  const int hx = __double2hiint(x);
  if (hx < 0x00100000 || hx >= 0x7ff00000) return log_outside(x);
  constexpr double kLn2Hi = 0.6931467056274414;      // ln 2 with the low 32 mantissa bits cleared
  constexpr double kLn2Lo = 4.7493250390316726e-07;  // ln 2 - kLn2Hi
  const int mb = hx & 0x000fffff;
  const int j = (mb + 0x1000) >> 13;
  const double y = __hiloint2double(mb | 0x3ff00000, __double2loint(x));
  const double* e = g_log_tab[j];
  const double r = fma(y, __ldg(e), -1.0);
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(r, q, 1.0 / 5.0);
  q = fma(r, q, -0.25);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  const double l1p = fma(r * r, q, r);  // ln(1 + r)
  const double md = (double)((hx >> 20) - 1023);
  const double t = fma(md, kLn2Hi, __ldg(e + 1));
  return t + fma(md, kLn2Lo, __ldg(e + 2) + l1p);
}

// 1/x by Newton's iteration r <- r + r (1 - x r) from the hardware's approximate
// reciprocal (two steps take its error below one ulp); magnitudes outside
// [2^-1000, 2^1000], zero, infinities and NaN take the IEEE division.
__device__ __forceinline__ double xrcp(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7ff;
  if (ex < 23 || ex > 2023) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}


// RODAS4 coefficients in constant memory (stages are indexed at run time).
static __constant__ double c_rodasA[6][6] = CHEM_RODAS_A;
static __constant__ double c_rodasC[6][6] = CHEM_RODAS_C;
static __constant__ double c_rodasM[6] = CHEM_RODAS_M;

// Method traits: stage count, step-size exponent 1/Q and the transformed coefficients.
// RODAS4 reads its published table from constant memory; the W-method reads the table
// the host converted from its published original form (kernel arguments).
template <int MTH>
struct Meth;
template <>
struct Meth<METHOD_RODAS4> {
  static constexpr int S = 6, Q = 4;
  static constexpr bool E_LAST = true;  // error estimate = last stage
  __device__ static double gamma(const IntegrateArgs&) { return kRodasGamma; }
  __device__ static double a(const IntegrateArgs&, int i, int j) { return c_rodasA[i][j]; }
  __device__ static double c(const IntegrateArgs&, int i, int j) { return c_rodasC[i][j]; }
  __device__ static double m(const IntegrateArgs&, int j) { return c_rodasM[j]; }
  __device__ static double e(const IntegrateArgs&, int) { return 0.0; }
};
template <>
struct Meth<METHOD_ROS34PW2> {
  static constexpr int S = 4, Q = 3;
  static constexpr bool E_LAST = false;
  __device__ static double gamma(const IntegrateArgs& g) { return g.tab.gamma; }
  __device__ static double a(const IntegrateArgs& g, int i, int j) { return g.tab.a[i][j]; }
  __device__ static double c(const IntegrateArgs& g, int i, int j) { return g.tab.c[i][j]; }
  __device__ static double m(const IntegrateArgs& g, int j) { return g.tab.m[j]; }
  __device__ static double e(const IntegrateArgs& g, int j) { return g.tab.e[j]; }
};

// Precision policy: LU = type of the factorised matrix, ASM = type the Jacobian is
// assembled in; IR = refine each solve against the assembled matrix.
template <int PREC>
struct Policy {
  using LU = double;
  using ASM = double;
  static constexpr bool IR = false;
};
template <>
struct Policy<PREC_MIXED> {
  using LU = float;
  using ASM = ff2;  // float-float: about 48 significant bits, on the FP32 pipe
  static constexpr bool IR = true;
};
template <>
struct Policy<PREC_FP32ASM> {
  using LU = float;
  using ASM = float;
  static constexpr bool IR = true;
};

// ---------------------------------------------------------------------------
// shared-memory carve-up
// ---------------------------------------------------------------------------
struct Layout {
  int nmax, ld;            // matrix dimension bound and leading dimension (odd)
  int Kmax, Imax;
  size_t off_vec, off_sp, off_rx, off_M, off_M0, off_piv, off_red, total;
};

__host__ __device__ inline int odd_ld(int n) { return n | 1; }

// vectors (double): y, yn, ys, f0, fv, rr, u[6], sc  -> 13 n
// species (double): C, hRT, cpR, eg, dcp, dk, akT, ek, ieg -> 9 K
// reactions (double): q, D, dTc, P, dqs[4] -> 8 I
// m0_global: the mixed form's assembled matrix lives in a global-memory slot of
// the CTA instead of shared memory (large mechanisms, persistent schedulers).
__host__ __device__ inline Layout make_layout(int Kmax, int Imax, int prec, bool m0_global = false) {
  Layout L;
  L.nmax = Kmax + 1;
  L.ld = odd_ld(L.nmax);
  L.Kmax = Kmax;
  L.Imax = Imax;
  size_t o = 0;
  L.off_red = o;
  o += 64 * sizeof(double);
  L.off_vec = o;
  o += (size_t)13 * L.nmax * sizeof(double);
  L.off_sp = o;
  o += (size_t)9 * Kmax * sizeof(double);
  L.off_rx = o;
  if (prec == PREC_FP64) {
    o += (size_t)8 * Imax * sizeof(double);
    L.off_M = o;
    o += (size_t)L.nmax * L.ld * sizeof(double);
  } else {
    // The FP32 factor matrix is written only after the assembly has consumed the
    // per-reaction Jacobian data (everything after q), so it shares their space.
    L.off_M = o + (size_t)Imax * sizeof(double);
    const size_t jac = (size_t)7 * Imax * sizeof(double);
    const size_t mat = (size_t)L.nmax * L.ld * sizeof(float);
    o += (size_t)Imax * sizeof(double) + (jac > mat ? jac : mat);
  }
  o = (o + 15) & ~(size_t)15;
  L.off_M0 = o;
  if (prec == PREC_MIXED && !m0_global) o += (size_t)L.nmax * L.ld * sizeof(double);
  if (prec == PREC_FP32ASM) o += (size_t)L.nmax * L.ld * sizeof(float);
  o = (o + 15) & ~(size_t)15;
  L.off_piv = o;
  o += (size_t)2 * L.nmax * sizeof(int);  // pivots, permutation
  o += (size_t)L.nmax * sizeof(double);   // inverse diagonal of U
  o = (o + 15) & ~(size_t)15;
  L.total = o;
  return L;
}


// Scalars kept in the reduction area (its first 32 slots are unused).
// SC_OUT: 8 broadcast results of Cta::reduce; SC_PIV: pivot search slots (12 NW bytes)
// (SC_INVT during the rate evaluation, SC_INVP during the LU: never live together)
enum { SC_OUT = 32, SC_LOGT = 48, SC_INVT = 49, SC_INVP = 49, SC_FLAG = 50, SC_MISC = 51, SC_PIV = 52 };

template <int NW>
struct Cta {
  static constexpr int NT = NW * 32;
  static constexpr int SW = NW - 1;  // the warp that computes CTA scalars (ln T, 1/T, the FP64 solve)
  int tid, lane, warp;
  double* red;
  // vectors
  double *y, *yn, *ys, *f0, *fv, *rr, *u, *sc;
  // species
  double *C, *hRT, *cpR, *eg, *dcp, *dk, *akT, *ek, *ieg;
  // reactions
  double *q, *D, *dTc, *P, *dqs;
  void* M;
  void* M0;
  int *piv, *perm;
  double* invd;

  __device__ void bind(unsigned char* base, const Layout& L) {
    tid = threadIdx.x;
    lane = tid & 31;
    warp = tid >> 5;
    red = reinterpret_cast<double*>(base + L.off_red);
    double* v = reinterpret_cast<double*>(base + L.off_vec);
    const int n = L.nmax;
    y = v;
    yn = v + n;
    ys = v + 2 * n;
    f0 = v + 3 * n;
    fv = v + 4 * n;
    rr = v + 5 * n;
    u = v + 6 * n;   // 6 n
    sc = v + 12 * n;
    double* s = reinterpret_cast<double*>(base + L.off_sp);
    const int K = L.Kmax;
    C = s;
    hRT = s + K;
    cpR = s + 2 * K;
    eg = s + 3 * K;
    dcp = s + 4 * K;
    dk = s + 5 * K;
    akT = s + 6 * K;
    ek = s + 7 * K;
    ieg = s + 8 * K;
    double* r = reinterpret_cast<double*>(base + L.off_rx);
    const int I = L.Imax;
    q = r;
    D = r + I;
    dTc = r + 2 * I;
    P = r + 3 * I;
    dqs = r + 4 * I;
    M = base + L.off_M;
    M0 = base + L.off_M0;
    piv = reinterpret_cast<int*>(base + L.off_piv);
    perm = piv + L.nmax;
    invd = reinterpret_cast<double*>(perm + L.nmax);
  }


  // Sum of NV (1, 2 or 4) values over the CTA; every thread receives the same
  // totals (fixed summation order: deterministic). Only the first nw warps may hold
  // non-zero values, nw = warps_for(count) of a loop over count <= n entries.
  // The FP64 pipe, shared by the SM's four schedulers, bounds the integration, so
  // the sum is arranged to issue few FP64 instructions:
  //  1. each data warp folds its NV values into one value per lane by log2(NV)
  //     transposing butterfly levels (a lane keeps one of two values and adds the
  //     partner's half of it), so that lane groups of 32/NV lanes carry one value each;
  //  2. warps 1..nw-1 leave their lane values in the scratch vector sc (free outside
  //     the solves; 32 (nw-1) <= count <= n entries), warp 0 adds them lane by lane;
  //  3. warp 0 finishes the butterfly inside each lane group and passes the totals to
  //     fin(tot, out), which derives NO scalars from them; lane 0's out[] reaches
  //     every thread through shared memory, so scalar follow-up work (reciprocals,
  //     roots) runs on one warp, not all.
  // With two data warps: 6, 7 and 10 FP64 warp instructions for 1, 2 and 4 values,
  // against 11, 22 and 44 for one shuffle tree per value and warp.
  template <int NV, int NO, class F>
  __device__ void reduce(const double (&v)[NV], int nw, F fin, double (&out)[NO]) {
    static_assert(NV == 1 || NV == 2 || NV == 4, "reduce: 1, 2 or 4 values");
    static_assert(NO <= 8, "reduction slots");
    constexpr int LV = NV == 1 ? 0 : (NV == 2 ? 1 : 2);  // transposing levels
    double x = 0.0;
    if (warp < nw) {
      if constexpr (NV == 1) {
        x = v[0];
      } else {
        // level 16: lanes 0-15 keep value 0 (and 2), lanes 16-31 value 1 (and 3)
        const bool h16 = lane & 16;
        x = (h16 ? v[1] : v[0]) + __shfl_xor_sync(FULLMASK, h16 ? v[0] : v[1], 16);
        if constexpr (NV == 4) {
          const double x2 = (h16 ? v[3] : v[2]) + __shfl_xor_sync(FULLMASK, h16 ? v[2] : v[3], 16);
          // level 8: lanes with bit 3 clear keep values 0/1, set keep 2/3
          const bool h8 = lane & 8;
          x = (h8 ? x2 : x) + __shfl_xor_sync(FULLMASK, h8 ? x : x2, 8);
        }
      }
      if (warp > 0) sc[(warp - 1) * 32 + lane] = x;
    }
    __syncthreads();
    if (warp == 0) {
      for (int w = 1; w < nw; ++w) x += sc[(w - 1) * 32 + lane];
#pragma unroll
      for (int o = 16 >> LV; o; o >>= 1) x += __shfl_xor_sync(FULLMASK, x, o);
      double tot[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        // value a's lane group: bit 4 = a & 1, bit 3 = a >> 1
        const int src = NV == 1 ? 0 : (((a & 1) << 4) | ((a >> 1) << 3));
        tot[a] = NV == 1 ? x : __shfl_sync(FULLMASK, x, src);
      }
      double o[NO];
      fin(tot, o);
      if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NO; ++b) red[SC_OUT + b] = o[b];
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NO; ++b) out[b] = red[SC_OUT + b];
  }

  // Plain CTA sum of NV values (nw as in reduce).
  template <int NV>
  __device__ void sum(double (&v)[NV], int nw) {
    reduce(v, nw, [](const double (&t)[NV], double (&o)[NV]) {
#pragma unroll
      for (int a = 0; a < NV; ++a) o[a] = t[a];
    }, v);
  }
};

// number of warps that hold data in a loop `for (i = tid; i < count; i += NT)`
template <int NW>
__device__ __forceinline__ int warps_for(int count) {
  const int w = (count + 31) >> 5;
  return w < NW ? w : NW;
}

// Cell-level scalars shared by all threads of the CTA (identical in every thread).
struct Scal {
  double T, invT, logT, rho, irho, Wbar, cpm, icpm, fT, dcpm, Scpw;
};

// ---------------------------------------------------------------------------
// thermo, rates, RHS and the per-reaction Jacobian data
// ---------------------------------------------------------------------------
// RHS of y = [T, Y] at constant p into f[0..K]. With JAC, also the data the
// Jacobian assembly needs: per reaction the slot derivatives dq/dC, dq/dT at
// fixed C, sum_k C_k dq/dC_k (D), and the third-body/falloff coefficient P of
// eff_j in dq/dC_j; per species d_k = sum_i nu_ki D_i and a_kT = sum nu dTc.
// BIG: the cell's T is below the mechanism's T_bigG, where some species may have
// |G/RT| > kBigGRT (very low T with large formation enthalpies): the reverse-rate
// ratio then takes one exponential of the summed exponent per reaction instead of
// the product of four species factors, whose partial products could overflow or
// underflow. A separate instantiation, so that the common path carries no trace of it.
// FF (the forms with FP32 factors): the third-body sums [M] in float-float, and the
// slot derivatives and P stored as float-float pairs for the assembly.
template <int NW, bool JAC, bool FF, bool BIG>
__device__ Scal eval_rhs_t(const DevMech& m, Cta<NW>& c, const double* y, double p, double* f) {
  constexpr int NT = NW * 32;
  const int K = m.K;
  Scal s;
  s.T = y[0];
  // the scalar warp: ln T and 1/T for every thread (read after the reduction's barriers)
  if (c.warp == Cta<NW>::SW) {
    const double lg = xlog(s.T);
    const double iT = xrcp(s.T);
    if (c.lane == 0) {
      c.red[SC_LOGT] = lg;
      c.red[SC_INVT] = iT;
    }
  }
  {
    double part[1] = {0.0};
    for (int k = c.tid; k < K; k += NT) part[0] += y[1 + k] * m.invW[k];
    double o[3];
    const double T = s.T;
    // (fin runs after the reduction's first barrier: 1/T is in shared memory by then)
    c.reduce(part, warps_for<NW>(K), [&](const double (&t)[1], double (&r)[3]) {
      const double Wbar = xrcp(t[0]);
      r[0] = Wbar;
      r[1] = p * c.red[SC_INVT] * Wbar * (1.0 / kRc);  // rho = p Wbar / (Rc T)
      r[2] = kRc * T * t[0] / p;                       // 1 / rho
    }, o);
    s.Wbar = o[0];
    s.rho = o[1];
    s.irho = o[2];
  }
  s.logT = c.red[SC_LOGT];
  s.invT = c.red[SC_INVT];
  const double T = s.T, invT = s.invT, logT = s.logT;
  // species: thermo, exp(G/RT), concentrations
  for (int k = c.tid; k < K; k += NT) {
    const double* a = m.nasa + 36 * k;
    a += (T < a[34]) ? 0 : 17;
    double cp = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    double h = a[5] + T * (a[6] + T * (a[7] + T * (a[8] + T * a[9]))) + a[10] * invT;
    double sr = a[11] * logT + T * (a[12] + T * (a[13] + T * (a[14] + T * a[15]))) + a[16];
    c.cpR[k] = cp;
    c.hRT[k] = h;
    const double g = h - sr;
    const double e = xexp(g);
    c.eg[k] = e;
    c.ieg[k] = xrcp(e);
    if (BIG) c.ek[k] = g;  // G/RT (the slot is the Jacobian assembly's, unused until then)
    const double Ck = s.rho * y[1 + k] * m.invW[k];
    c.C[k] = Ck;
    // float-float copy of C for the third-body sums (the slot of d_k, which the
    // Jacobian evaluation writes only after the reaction loop)
    if (FF) reinterpret_cast<ff2*>(c.dk)[k] = ff_split(Ck);
    if (JAC) c.dcp[k] = a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]));
    // without Jacobian data the reverse term needs only C_k exp(G_k/RT) (the dcp slot)
    if (!JAC && !BIG) c.dcp[k] = Ck * e;
  }
  __syncthreads();
  const double cRT = kRc * T / kP0;  // (P0 / (Rc T))^-1
  const double icRT = kP0 * invT / kRc;
  // 32-reaction chunks of one kind each, dealt to the warps by estimated work
  const int* cs = m.chunk_sched[NW == 2 ? 0 : NW == 4 ? 1 : 2];
  for (int pos = cs[c.warp]; pos < cs[c.warp + 1]; ++pos) {
    const int i = cs[NW + 1 + pos] * 32 + c.lane;
    const int4 sl = m.slots[i];
    if (sl.x < 0) {  // null padding reaction
      c.q[i] = 0.0;
      if (JAC) {
        c.D[i] = c.dTc[i] = c.P[i] = 0.0;
        c.dqs[4 * i] = c.dqs[4 * i + 1] = c.dqs[4 * i + 2] = c.dqs[4 * i + 3] = 0.0;
      }
      continue;
    }
    const double* arp = m.arr + 4 * i;
    const double2 a01 = reinterpret_cast<const double2*>(arp)[0];
    const double2 a23 = reinterpret_cast<const double2*>(arp)[1];
    const struct { double x, y, z, w; } ar = {a01.x, a01.y, a23.x, a23.y};
    double kf = xexp(ar.x + ar.y * logT - ar.z * invT);
    const double Ca = c.C[sl.x];
    const double Cb = sl.y >= 0 ? c.C[sl.y] : 1.0;
    const double Cc = c.C[sl.z];
    const double Cd = sl.w >= 0 ? c.C[sl.w] : 1.0;
    const double Pf = Ca * Cb, Pb = Cc * Cd;
    // 1/Kc = exp(dG/RT) (Rc T/P0)^dnu with exp(dG/RT) from the species factors
    // (formed here only where kr itself is needed: Jacobian data, large-|G/RT| path)
    constexpr bool FAST = !JAC && !BIG;
    double ratio = 0.0;
    const int rv = m.rev[i];
    if (!FAST && (rv & 1)) {
      if (!BIG) {
        ratio = c.eg[sl.z] * c.ieg[sl.x];
        if (sl.w >= 0) ratio *= c.eg[sl.w];
        if (sl.y >= 0) ratio *= c.ieg[sl.y];
        ratio *= (rv >> 1) == 2 ? cRT : (rv >> 1) == 0 ? icRT : 1.0;
      } else {
        double dg = c.ek[sl.z] - c.ek[sl.x];
        if (sl.w >= 0) dg += c.ek[sl.w];
        if (sl.y >= 0) dg -= c.ek[sl.y];
        const double lc = logT + kLnRcP0;  // ln(Rc T / P0)
        dg += (rv >> 1) == 2 ? lc : (rv >> 1) == 0 ? -lc : 0.0;
        ratio = xexp(dg);
      }
    }
    double Mc = 0.0, phi = 1.0;
    double dk_dM = 0.0, dlnk = (ar.y + ar.z * invT) * invT, dk_dT = 0.0;
    if (i >= m.i_tb0) {
      // efficiencies species-major: the warp's 32 reactions read one row per species
      const int r = i - m.i_tb0, ntb = m.n_tb;
      if (FF) {
        const ff2* ef = m.effT_ff + r;
        const ff2* Cf = reinterpret_cast<const ff2*>(c.dk);
        ff2 acc = {0.0f, 0.0f};
        for (int k = 0; k < K; ++k) acc = ff_fma(ef[(size_t)k * ntb], Cf[k], acc);
        Mc = ff_value(acc);
      } else {
        const double* e = m.effT + r;
        for (int k = 0; k < K; ++k) Mc += e[(size_t)k * ntb] * c.C[k];
      }
      if (i < m.i_fo0) phi = Mc;
    }
    if (i >= m.i_fo0) {
      // fo[0..2] hold the low-pressure minus the high-pressure Arrhenius parameters,
      // so one exponential gives k0 / kinf
      const double* fo = m.fo + 8 * (i - m.i_fo0);
      const double r0 = xexp(fo[0] + fo[1] * logT - fo[2] * invT);  // k0 / kinf
      const double Pr = r0 * Mc;
      double F = 1.0, dlgF_dL = 0.0, dlnF_dT = 0.0;
      if (i >= m.i_troe0) {
        const double alpha = fo[3];
        // fo[4] = 1/T***, fo[5] = 1/T*
        const double e3 = xexp(-T * fo[4]), e1 = xexp(-T * fo[5]);
        double Fc = (1.0 - alpha) * e3 + alpha * e1;
        double dFc = -(1.0 - alpha) * fo[4] * e3 - alpha * fo[5] * e1;
        if (fo[6] > 0.0) {
          const double e2 = xexp(-fo[6] * invT);
          Fc += e2;
          dFc += fo[6] * invT * invT * e2;
        }
        const double lF = xlog(Fc) * kInvLn10;
        const double cc = -0.4 - 0.67 * lF, nn = 0.75 - 1.27 * lF;
        const double x = xlog(Pr) * kInvLn10 + cc;
        const double iden = xrcp(nn - 0.14 * x);
        const double f1 = x * iden;
        const double ig = xrcp(fma(f1, f1, 1.0));
        const double lgF = lF * ig;
        F = xexp(lgF * 2.302585092994046);  // 10^lgF
        if (JAC) {
          // partial derivatives of log10 F by log10 Pr and by log10 Fc
          const double df1_dL = nn * iden * iden;
          const double df1_dlF = (-0.67 - f1 * (-1.27 + 0.14 * 0.67)) * iden;
          dlgF_dL = -2.0 * lgF * ig * f1 * df1_dL;
          const double dlgF_dlF = ig - 2.0 * lgF * ig * f1 * df1_dlF;
          dlnF_dT = dlgF_dlF * dFc * xrcp(Fc);  // d ln F / dT at fixed Pr
        }
      }
      const double red1 = xrcp(1.0 + Pr);
      const double kinf = kf;
      kf = kinf * Pr * red1 * F;
      if (JAC) {
        // d ln k / d ln Pr = 1/(1 + Pr) + d log10 F / d log10 Pr; Pr = (k0/kinf) [M]
        const double g = red1 + dlgF_dL;
        dk_dM = kinf * red1 * F * g * r0;
        dk_dT = kf * (dlnk + g * (fo[1] + fo[2] * invT) * invT + dlnF_dT);
      }
    }
    const double kr = kf * ratio;
    double net;
    if constexpr (FAST) {
      // kr Pb = kf c / (e_x e_y) (C_z e_z)(C_w e_w), e = exp(G/RT), c = (Rc T/P0)^dnu:
      // q = kf (Pf - u rb) with u = c / (e_x e_y), rb = (C e)_z (C e)_w; plain
      // third-body chunks multiply by [M], the other kinds (phi = 1) skip it
      net = kf * Pf;
      if (rv & 1) {
        double ri = c.ieg[sl.x];
        if (sl.y >= 0) ri *= c.ieg[sl.y];
        double rb = c.dcp[sl.z];
        if (sl.w >= 0) rb *= c.dcp[sl.w];
        const double u = ri * ((rv >> 1) == 2 ? cRT : (rv >> 1) == 0 ? icRT : 1.0);
        net = kf * fma(-u, rb, Pf);
      }
      c.q[i] = (i >= m.i_tb0 && i < m.i_fo0) ? phi * net : net;
    } else {
      net = kf * Pf - kr * Pb;
      c.q[i] = phi * net;
    }
    if (JAC) {
      // d ln Kc / dT = dH/(R T^2) - dnu/T
      double dH = c.hRT[sl.z] + (sl.w >= 0 ? c.hRT[sl.w] : 0.0) - c.hRT[sl.x] -
                  (sl.y >= 0 ? c.hRT[sl.y] : 0.0);
      const double dlnKc = (dH - ar.w) * invT;
      double dq[4];
      dq[0] = phi * kf * Cb;
      dq[1] = sl.y >= 0 ? phi * kf * Ca : 0.0;
      dq[2] = -phi * kr * Cd;
      dq[3] = sl.w >= 0 ? -phi * kr * Cc : 0.0;
      if (FF) {
        // the float-float assembly's copy (hi, lo), split once here
        ff2* dqf = reinterpret_cast<ff2*>(c.dqs) + 4 * i;
        dqf[0] = ff_split(dq[0]);
        dqf[1] = sl.y >= 0 ? ff_split(dq[1]) : ff2{0.0f, 0.0f};
        dqf[2] = ff_split(dq[2]);
        dqf[3] = sl.w >= 0 ? ff_split(dq[3]) : ff2{0.0f, 0.0f};
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) c.dqs[4 * i + u] = dq[u];
      }
      double Dsum = Ca * dq[0] + (sl.y >= 0 ? Cb * dq[1] : 0.0) + Cc * dq[2] + (sl.w >= 0 ? Cd * dq[3] : 0.0);
      double dtc, Pc;
      if (i >= m.i_fo0) {
        const double netc = Pf - ratio * Pb;
        dtc = dk_dT * netc + ((rv & 1) ? kr * Pb * dlnKc : 0.0);
        Pc = dk_dM * netc;
      } else {
        const double dkf = kf * dlnk;
        const double dkr = kr * (dlnk - dlnKc);
        dtc = phi * (dkf * Pf - dkr * Pb);
        Pc = (i >= m.i_tb0) ? net : 0.0;
      }
      if (i >= m.i_tb0) Dsum += Mc * Pc;
      c.dTc[i] = dtc;
      if (FF)
        reinterpret_cast<ff2*>(c.P)[i] = ff_split(Pc);
      else
        c.P[i] = Pc;
      c.D[i] = Dsum;
    }
  }
  __syncthreads();
  // species: production rates, f_k, enthalpy and heat-capacity sums
  double part[JAC ? 4 : 2];
  part[0] = part[1] = 0.0;
  if (JAC) part[2] = part[3] = 0.0;
  for (int k = c.tid; k < K; k += NT) {
    double w = 0.0, dd = 0.0, at = 0.0;
    for (int e = m.sp_ptr[k]; e < m.sp_ptr[k + 1]; ++e) {
      const int2 en = m.sp_ent[e];
      const double nu = m.sp_nu[e];
      w += nu * c.q[en.x];
      if (JAC) {
        dd += nu * c.D[en.x];
        at += nu * c.dTc[en.x];
      }
    }
    f[1 + k] = m.W[k] * w * s.irho;
    part[0] += c.hRT[k] * w;                  // Qh / (Rc T)
    part[1] += y[1 + k] * c.cpR[k] * m.invW[k];  // cpm / Rc
    if (JAC) {
      c.dk[k] = dd;
      c.akT[k] = at;
      part[2] += y[1 + k] * c.dcp[k] * m.invW[k];  // dcpm/dT / Rc
      part[3] += c.cpR[k] * w;                      // sum cp_k omega_k / Rc
    }
  }
  {
    double o[5];
    const double T = s.T, irho = s.irho;
    c.reduce(part, warps_for<NW>(K), [&](const double (&t)[JAC ? 4 : 2], double (&r)[5]) {
      const double cpm = kRc * t[1];
      const double icpm = xrcp(cpm);
      const double fT = -kRc * T * t[0] * irho * icpm;  // -Qh / (rho cp), Qh = Rc T sum hRT_k w_k
      r[0] = cpm;
      r[1] = icpm;
      r[2] = fT;
      if constexpr (JAC) {
        r[3] = kRc * t[2];
        r[4] = kRc * t[3];
      } else {
        r[3] = r[4] = 0.0;
      }
      if (c.lane == 0) f[0] = fT;  // visible after the reduction's last barrier
    }, o);
    s.cpm = o[0];
    s.icpm = o[1];
    s.fT = o[2];
    s.dcpm = o[3];
    s.Scpw = o[4];
  }
  return s;
}

template <int NW, bool JAC, bool FF>
__device__ __noinline__ Scal eval_rhs_big(const DevMech& m, Cta<NW>& c, const double* y, double p, double* f) {
  return eval_rhs_t<NW, JAC, FF, true>(m, c, y, p, f);
}

// RHS (and with JAC the Jacobian data) of the state y; T = y[0] selects the path.
template <int NW, bool JAC, bool FF = false>
__device__ __forceinline__ Scal eval_rhs(const DevMech& m, Cta<NW>& c, const double* y, double p, double* f) {
  if (y[0] < m.T_bigG) return eval_rhs_big<NW, JAC, FF>(m, c, y, p, f);
  return eval_rhs_t<NW, JAC, FF, false>(m, c, y, p, f);
}

// ---------------------------------------------------------------------------
// Jacobian assembly (precision R) from the data of eval_rhs<JAC=true>.
// With A_kj = sum_i nu_ki dq_i/dC_j (mass-action slot terms plus the third-body /
// falloff term nu_ki P_i eff_ij), the species rows of the Jacobian are
//   J_kj = (W_k / W_j) (A_kj - (Wbar/rho) d_k) + f_k Wbar / W_j,
// so with sg = -1 for the iteration matrix M = I/(h gamma) - J (rf = 1/(h gamma))
// and sg = +1, rf = 0 for the Jacobian itself (JO), the stored value is
//   S_kj = B_kj / W_j + rf delta_kj,  B_kj = sg W_k A_kj + beta_k,
//   beta_k = sg (f_k Wbar - W_k (Wbar/rho) d_k).
// (1) species pass: e_k = h_k / (W_k cp), beta_k, the temperature column
//     J_k0 = (W_k/rho)(a_kT - d_k/T) + f_k/T; and the mass-action pair sums
//     sum sg nu_ki W_k dq_i/dC_j on the thread-balanced schedule, stored in place;
// (2) one warp per row: beta + pair sum, the dense third-body part in registers
//     (lane l holds columns l + 32 u), scaled by 1/W_j;
// (3) temperature row from column sums of the stored rows:
//     J_0j = -sum_k e_k J_kj - f_T cp_j/(W_j cp),
//     J_00 = -sum_k e_k J_k0 - sum_k cp_k omega_k/(rho cp) - f_T cp'/cp.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R fmaR(R a, R b, R c) {
  if constexpr (std::is_same<R, float>::value) return fmaf(a, b, c);
  else return fma(a, b, c);
}

// FFD: the per-reaction data (dq/dC, P) is stored as float-float pairs (the forms
// with FP32 factors); R = float then reads their hi parts.
template <bool FFD>
__device__ __forceinline__ double rx_data(const double* a, int i) {
  if constexpr (FFD) return (double)reinterpret_cast<const ff2*>(a)[i].hi;
  else return a[i];
}

template <int NW, class R, bool JO, int U, bool FFD>
__device__ void assemble_rows(const DevMech& m, Cta<NW>& c, R* A, int K, int ld, R rf) {
  constexpr double SG = JO ? 1.0 : -1.0;
  for (int k = c.warp; k < K; k += NW) {
    R* row = A + (1 + k) * ld + 1;
    const R beta = R(c.akT[k]);
    R acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned msk = m.jmask[k * U + u];
      acc[u] = ((msk >> c.lane) & 1u) ? beta + row[c.lane + 32 * u] : beta;
    }
    // third-body / falloff part: 32 row coefficients sg nu_ki W_k P_i at a time,
    // broadcast from their lanes
    const int t1 = m.tr_ptr[k + 1];
    for (int tb = m.tr_ptr[k]; tb < t1; tb += 32) {
      const int t = tb + c.lane;
      R cl = R(0);
      int rl = 0;
      if (t < t1) {
        const int ri = m.tr_ent[t].x;
        cl = R(SG * m.tr_nu[t] * rx_data<FFD>(c.P, ri));
        rl = ri - m.i_tb0;
      }
      const int cnt = min(32, t1 - tb);
      for (int q = 0; q < cnt; ++q) {
        const R coef = __shfl_sync(FULLMASK, cl, q);
        const double* e = m.eff + (size_t)__shfl_sync(FULLMASK, rl, q) * K;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = c.lane + 32 * u;
          if (u < U - 1 || j < K) acc[u] = fmaR(coef, R(e[j]), acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = c.lane + 32 * u;
      if (u < U - 1 || j < K) row[j] = fmaR(acc[u], R(m.invW[j]), j == k ? rf : R(0));
    }
  }
}

template <int NW, class R, bool JO, bool FFD = false>
__device__ void assemble(const DevMech& m, Cta<NW>& c, const Scal& s, const double* f, double fac, void* target) {
  constexpr int NT = NW * 32;
  constexpr double SG = JO ? 1.0 : -1.0;
  const int K = m.K, n = K + 1, ld = odd_ld(n);
  R* A = reinterpret_cast<R*>(target);
  const R rf = JO ? R(0) : R(fac);
  // (1) species pass
  const double eT = kRc * s.T * s.icpm, wr = s.Wbar * s.irho;
  for (int k = c.tid; k < K; k += NT) {
    c.ek[k] = c.hRT[k] * eT * m.invW[k];
    const double Wk = m.W[k], dk = c.dk[k], fk = f[1 + k];
    A[(1 + k) * ld] = R(SG * (Wk * s.irho * (c.akT[k] - dk * s.invT) + fk * s.invT));
    c.akT[k] = SG * (fk * s.Wbar - Wk * wr * dk);  // beta_k (a_kT is consumed)
  }
  {
    const int v = NT == 64 ? 0 : NT == 128 ? 1 : 2;
    const int2* se = m.js_ent[v] + c.tid;
    const double* sn = m.js_nu[v] + c.tid;
    const int rounds = m.js_rounds[v];
    R a = R(0);
    for (int r = 0; r < rounds; ++r) {
      const int2 e = se[r * NT];
      if (e.x >= 0) a = fmaR(R(SG * sn[r * NT]), R(rx_data<FFD>(c.dqs, e.x)), a);
      if (e.y >= 0) {
        A[e.y] = a;
        a = R(0);
      }
    }
  }
  __syncthreads();
  // (2) species rows
  switch ((K + 31) >> 5) {
    case 1: assemble_rows<NW, R, JO, 1, FFD>(m, c, A, K, ld, rf); break;
    case 2: assemble_rows<NW, R, JO, 2, FFD>(m, c, A, K, ld, rf); break;
    case 3: assemble_rows<NW, R, JO, 3, FFD>(m, c, A, K, ld, rf); break;
    case 4: assemble_rows<NW, R, JO, 4, FFD>(m, c, A, K, ld, rf); break;
    case 5: assemble_rows<NW, R, JO, 5, FFD>(m, c, A, K, ld, rf); break;
    case 6: assemble_rows<NW, R, JO, 6, FFD>(m, c, A, K, ld, rf); break;
    case 7: assemble_rows<NW, R, JO, 7, FFD>(m, c, A, K, ld, rf); break;
    default: assemble_rows<NW, R, JO, 8, FFD>(m, c, A, K, ld, rf); break;
  }
  __syncthreads();
  // (3) temperature row; with acc = sum_k e_k S_kj, sum_k e_k J_kj = sg (acc - rf e_(j-1)),
  //     so S_0j = rf e_(j-1) - acc - sg extra_j (j >= 1) and S_00 = rf - acc - sg extra_0
  const double ft = s.fT * s.icpm;
  for (int j = NT - 1 - c.tid; j < n; j += NT) {  // from the last warp down, as the residual rows
    R acc = R(0);
    for (int k = 0; k < K; ++k) acc = fmaR(R(c.ek[k]), A[(1 + k) * ld + j], acc);
    R v;
    if (j == 0)
      v = rf - acc - R(SG * (s.Scpw * s.irho * s.icpm + ft * s.dcpm));
    else
      v = rf * R(c.ek[j - 1]) - acc - R(SG * ft * c.cpR[j - 1] * kRc * m.invW[j - 1]);
    A[j] = v;
  }
  __syncthreads();
}

// The same assembly in float-float arithmetic (the mixed form): the same terms in the
// same order, from float-float copies of the per-reaction data (dq/dC and P, split
// once by eval_rhs) and of the mechanism's constants (1/W, nu W, efficiencies), so
// that every sum and product of the pass runs on the FP32 pipe; the species-level
// scalars are formed in FP64 and split once per species. A holds (hi, lo) per entry;
// its error is a few units of 2^-48 relative to the sums' terms, far below the FP32
// factorisation's, so the refinement converges to the same solutions.
template <int NW, bool JO, int U>
__device__ void assemble_rows_ff(const DevMech& m, Cta<NW>& c, ff2* A, int K, int ld, ff2 rf) {
  const ff2* beta_ff = reinterpret_cast<const ff2*>(c.akT);
  const ff2* Pf = reinterpret_cast<const ff2*>(c.P);
  const ff2 zero = {0.0f, 0.0f};
  for (int k = c.warp; k < K; k += NW) {
    ff2* row = A + (1 + k) * ld + 1;
    const ff2 beta = beta_ff[k];
    ff_sum acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned msk = m.jmask[k * U + u];
      acc[u] = ff_sum(beta);
      if ((msk >> c.lane) & 1u) acc[u].add(row[c.lane + 32 * u]);
    }
    const int t1 = m.tr_ptr[k + 1];
    for (int tb = m.tr_ptr[k]; tb < t1; tb += 32) {
      const int t = tb + c.lane;
      ff2 cl = zero;
      int rl = 0;
      if (t < t1) {
        const int ri = m.tr_ent[t].x;
        const ff2 tn = m.tr_nu_ff[t];
        cl = ff_mul(JO ? tn : ff_neg(tn), Pf[ri]);
        rl = ri - m.i_tb0;
      }
      const int cnt = min(32, t1 - tb);
      for (int q = 0; q < cnt; ++q) {
        const ff2 coef = {__shfl_sync(FULLMASK, cl.hi, q), __shfl_sync(FULLMASK, cl.lo, q)};
        const ff2* e = m.eff_ff + (size_t)__shfl_sync(FULLMASK, rl, q) * K;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = c.lane + 32 * u;
          if (u < U - 1 || j < K) acc[u].add_prod(coef, e[j]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = c.lane + 32 * u;
      if (u < U - 1 || j < K) row[j] = ff_fma(acc[u].value(), m.invW_ff[j], j == k ? rf : zero);
    }
  }
}

template <int NW, bool JO>
__device__ void assemble_ff(const DevMech& m, Cta<NW>& c, const Scal& s, const double* f, double fac, ff2* A) {
  constexpr int NT = NW * 32;
  constexpr double SG = JO ? 1.0 : -1.0;
  const int K = m.K, n = K + 1, ld = odd_ld(n);
  const ff2 zero = {0.0f, 0.0f};
  const ff2 rf = JO ? zero : ff_split(fac);
  ff2* ek = reinterpret_cast<ff2*>(c.ek);
  ff2* beta = reinterpret_cast<ff2*>(c.akT);
  const ff2* dq = reinterpret_cast<const ff2*>(c.dqs);
  // (1) species pass
  const double eT = kRc * s.T * s.icpm, wr = s.Wbar * s.irho;
  for (int k = c.tid; k < K; k += NT) {
    ek[k] = ff_split(c.hRT[k] * eT * m.invW[k]);
    const double Wk = m.W[k], dk = c.dk[k], fk = f[1 + k];
    A[(1 + k) * ld] = ff_split(SG * (Wk * s.irho * (c.akT[k] - dk * s.invT) + fk * s.invT));
    beta[k] = ff_split(SG * (fk * s.Wbar - Wk * wr * dk));  // beta_k (a_kT is consumed)
  }
  {
    const int v = NT == 64 ? 0 : NT == 128 ? 1 : 2;
    const int2* se = m.js_ent[v] + c.tid;
    const ff2* sn = m.js_nu_ff[v] + c.tid;
    const int rounds = m.js_rounds[v];
    ff_sum a;
    for (int r = 0; r < rounds; ++r) {
      const int2 e = se[r * NT];
      if (e.x >= 0) {
        const ff2 w = sn[r * NT];
        a.add_prod(JO ? w : ff_neg(w), dq[e.x]);
      }
      if (e.y >= 0) {
        A[e.y] = a.value();
        a = ff_sum();
      }
    }
  }
  __syncthreads();
  // (2) species rows
  switch ((K + 31) >> 5) {
    case 1: assemble_rows_ff<NW, JO, 1>(m, c, A, K, ld, rf); break;
    case 2: assemble_rows_ff<NW, JO, 2>(m, c, A, K, ld, rf); break;
    case 3: assemble_rows_ff<NW, JO, 3>(m, c, A, K, ld, rf); break;
    case 4: assemble_rows_ff<NW, JO, 4>(m, c, A, K, ld, rf); break;
    case 5: assemble_rows_ff<NW, JO, 5>(m, c, A, K, ld, rf); break;
    case 6: assemble_rows_ff<NW, JO, 6>(m, c, A, K, ld, rf); break;
    case 7: assemble_rows_ff<NW, JO, 7>(m, c, A, K, ld, rf); break;
    default: assemble_rows_ff<NW, JO, 8>(m, c, A, K, ld, rf); break;
  }
  __syncthreads();
  // (3) temperature row, as in assemble()
  const double ft = s.fT * s.icpm;
  for (int j = NT - 1 - c.tid; j < n; j += NT) {
    ff_sum sum;
    for (int k = 0; k < K; ++k) sum.add_prod(ek[k], A[(1 + k) * ld + j]);
    const ff2 acc = sum.value();
    ff2 v;
    if (j == 0)
      v = ff_sub(ff_sub(rf, acc), ff_split(SG * (s.Scpw * s.irho * s.icpm + ft * s.dcpm)));
    else
      v = ff_sub(ff_sub(ff_mul(rf, ek[j - 1]), acc), ff_split(SG * ft * c.cpR[j - 1] * kRc * m.invW[j - 1]));
    A[j] = v;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Pivot candidates: every warp writes (max |value|, lowest row index) of its rows;
// every thread then reduces the NW partials in the same order (same result).
// ---------------------------------------------------------------------------
template <int NW>
__device__ __forceinline__ int pivot_reduce(Cta<NW>& c, float* pmax, int* pidx, int n) {
  float best = -1.0f;
  int bi = n;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const float v = pmax[w];
    const int i = pidx[w];
    if (v > best || (v == best && i < bi)) { best = v; bi = i; }
  }
  return bi;
}

// Warp-level (value, index) maximum with the lowest index on ties; lane 0 stores it.
__device__ __forceinline__ void warp_argmax_store(float v, int i, int lane, float* pmax, int* pidx, int warp) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float ov = __shfl_xor_sync(FULLMASK, v, o);
    const int oi = __shfl_xor_sync(FULLMASK, i, o);
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
  }
  if (lane == 0) {
    pmax[warp] = v;
    pidx[warp] = i;
  }
}

// ---------------------------------------------------------------------------
// dense LU with partial pivoting (row interchange to the largest |a_ik|, lowest
// row index on ties; the pivot choice compares magnitudes rounded to FP32), in
// place; the search for the next pivot is fused into the elimination, so each
// column costs two CTA barriers. Then the composed row permutation and the
// inverse diagonal of U for the solves. Returns 0 or 1 + k for a zero pivot.
// ---------------------------------------------------------------------------
template <int NW, class R>
__device__ int lu_factor(Cta<NW>& c, R* a, int n, bool pivot = true) {
  constexpr int NT = NW * 32;
  const int ld = odd_ld(n);
  float* pmax = reinterpret_cast<float*>(c.red + SC_PIV);
  int* pidx = reinterpret_cast<int*>(c.red + SC_PIV + NW);
  double* spinv = c.red + SC_INVP;
  int info = 0;
  // candidates for column 0
  {
    float v = -1.0f;
    int bi = n;
    for (int i = c.tid; i < n; i += NT) {
      const float x = fabsf((float)a[i * ld]);
      if (x > v || (x == v && i < bi)) { v = x; bi = i; }
    }
    warp_argmax_store(v, bi, c.lane, pmax, pidx, c.warp);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    int p = pivot ? pivot_reduce<NW>(c, pmax, pidx, n) : k;  // no pivoting: the diagonal
    if (p >= n) p = k;  // a column of NaN: the zero-pivot path below
    if (c.tid == 0) {
      c.piv[k] = p;
      const double pv = (double)a[p * ld + k];
      spinv[0] = pv != 0.0 && isfinite(pv) ? 1.0 / pv : 0.0;
    }
    if (p != k)
      for (int j = c.tid; j < n; j += NT) {
        const R t = a[k * ld + j];
        a[k * ld + j] = a[p * ld + j];
        a[p * ld + j] = t;
      }
    __syncthreads();
    const R invp = R(spinv[0]);
    if (invp == R(0) && info == 0) info = k + 1;
    float v = -1.0f;
    int bi = n;
    for (int i = k + 1 + c.warp; i < n; i += NW) {
      const R l = a[i * ld + k] * invp;
      __syncwarp();
      if (c.lane == 0) a[i * ld + k] = l;
      for (int j = k + 1 + c.lane; j < n; j += 32) {
        const R nv = a[i * ld + j] - l * a[k * ld + j];
        a[i * ld + j] = nv;
        if (j == k + 1) {
          const float x = fabsf((float)nv);
          if (x > v || (x == v && i < bi)) { v = x; bi = i; }
        }
      }
    }
    warp_argmax_store(v, bi, c.lane, pmax, pidx, c.warp);
    __syncthreads();
  }
  // composed permutation: position i of the pivoted system holds original row perm[i]
  if (c.tid == 0) {
    for (int i = 0; i < n; ++i) c.perm[i] = i;
    for (int k = 0; k < n; ++k) {
      const int p = c.piv[k];
      const int t = c.perm[k];
      c.perm[k] = c.perm[p];
      c.perm[p] = t;
    }
  }
  for (int i = c.tid; i < n; i += NT) c.invd[i] = 1.0 / (double)a[i * ld + i];
  __syncthreads();
  return info;
}

// Forward/back substitution by one warp, in place on x (already permuted).
template <class R>
__device__ void lu_solve_warp(const R* a, int n, const double* invd, R* x, int lane) {
  const int ld = odd_ld(n);
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const int jend = min(i0 + 32, n);
    R xi = i < n ? x[i] : R(0);
    for (int j = i0; j < jend; ++j) {
      const R xj = __shfl_sync(FULLMASK, xi, j - i0);
      if (i > j && i < n) xi -= a[i * ld + j] * xj;
    }
    if (i < n) x[i] = xi;
    __syncwarp();
    for (int r = i0 + 32 + lane; r < n; r += 32) {
      R sacc = R(0);
      for (int j = i0; j < jend; ++j) sacc += a[r * ld + j] * x[j];
      x[r] -= sacc;
    }
    __syncwarp();
  }
  for (int i1 = n; i1 > 0; i1 -= 32) {
    const int i0 = max(0, i1 - 32);
    const int i = i0 + lane;
    R xi = i < i1 ? x[i] : R(0);
    for (int j = i1 - 1; j >= i0; --j) {
      if (i == j) xi *= R(invd[j]);
      const R xj = __shfl_sync(FULLMASK, xi, j - i0);
      if (i < j) xi -= a[i * ld + j] * xj;
    }
    if (i < i1) x[i] = xi;
    __syncwarp();
    for (int r = lane; r < i0; r += 32) {
      R sacc = R(0);
      for (int j = i0; j < i1; ++j) sacc += a[r * ld + j] * x[j];
      x[r] -= sacc;
    }
    __syncwarp();
  }
}

// In-place Gauss-Jordan inverse (FP32) with partial pivoting: row interchange to
// the largest |a_ik| (lowest row index on ties), the normalised pivot row kept in a
// copy while every other row is eliminated (the next pivot search is fused into
// that elimination: two CTA barriers per column); the inverse is completed by the
// column interchanges in reverse order. Returns 0 or 1 + k for a zero pivot.
template <int NW>
__device__ int gj_invert(Cta<NW>& c, float* a, int n) {
  constexpr int NT = NW * 32;
  const int ld = odd_ld(n);
  float* pmax = reinterpret_cast<float*>(c.red + SC_PIV);
  int* pidx = reinterpret_cast<int*>(c.red + SC_PIV + NW);
  float* pr = reinterpret_cast<float*>(c.rr);  // normalised pivot row
  int info = 0;
  {
    float v = -1.0f;
    int bi = n;
    for (int i = c.tid; i < n; i += NT) {
      const float x = fabsf(a[i * ld]);
      if (x > v || (x == v && i < bi)) { v = x; bi = i; }
    }
    warp_argmax_store(v, bi, c.lane, pmax, pidx, c.warp);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    int p = pivot_reduce<NW>(c, pmax, pidx, n);
    if (p >= n) p = k;
    const float pv = a[p * ld + k];
    const float pinv = (pv != 0.0f && isfinite(pv)) ? 1.0f / pv : 0.0f;
    if (pinv == 0.0f && info == 0) info = k + 1;
    if (c.tid == 0) c.piv[k] = p;
    // interchange rows k and p; the new row k, normalised, goes to the copy
    for (int j = c.tid; j < n; j += NT) {
      const float rk = a[k * ld + j], rp = a[p * ld + j];
      if (p != k) a[p * ld + j] = rk;
      pr[j] = (j == k ? 1.0f : rp) * pinv;
    }
    __syncthreads();
    const int cn = k + 1;              // next pivot column
    const int own = cn & 31;           // lane owning column cn in the loops below
    float v = -1.0f;
    int bi = n;
    for (int i = c.warp; i < n; i += NW) {
      if (i == k) {
        for (int j = c.lane; j < n; j += 32) a[k * ld + j] = pr[j];
        continue;
      }
      const float fct = a[i * ld + k];
      __syncwarp();
      for (int j = c.lane; j < n; j += 32) {
        const float nv = (j == k ? 0.0f : a[i * ld + j]) - fct * pr[j];
        a[i * ld + j] = nv;
        if (j == cn && i > k) {
          const float x = fabsf(nv);
          if (x > v || (x == v && i < bi)) { v = x; bi = i; }
        }
      }
    }
    (void)own;
    warp_argmax_store(v, bi, c.lane, pmax, pidx, c.warp);
    __syncthreads();
  }
  // column interchanges in reverse order; each thread owns whole rows
  for (int i = c.tid; i < n; i += NT)
    for (int k = n - 1; k >= 0; --k) {
      const int p = c.piv[k];
      if (p != k) {
        const float t = a[i * ld + k];
        a[i * ld + k] = a[i * ld + p];
        a[i * ld + p] = t;
      }
    }
  __syncthreads();
  return info;
}

// Gauss-Jordan inverse (FP32) with the matrix in registers, by columns: warp w owns
// the columns j = w + NW c (c < CC), lane l the rows l + 32 s (s < RS). Partial
// pivoting by index (the unused row with the largest |a_ik|, lowest row index on
// ties; rows are not moved, the k-th pivot row is recorded instead). The warp
// owning column k searches it, publishes the pivot row p, 1/a_pk and the column (the multipliers) through
// shared memory (double-buffered), and every warp then broadcasts the pivot row's
// values of its own columns by warp shuffles and updates them: one CTA barrier per
// column. Column k is first replaced by the unit vector e_p, so it ends up holding
// column k of the inverse (in-place Gauss-Jordan). The inverse is written back as
// inv[Pinv[i]][P[j]] = W[i][j] (P = pivot rows in step order). Requires n <= 32 RS
// and n <= NW CC. Returns 0 or 1 + k for a zero pivot.
template <int NW, int RS, int CC>
__device__ int gj_invert_wc(Cta<NW>& c, float* A, int n) {
  const int ld = odd_ld(n);
  const int lane = c.lane, wp = c.warp;
  float* pcol = reinterpret_cast<float*>(c.u);          // [2][n] multipliers (u: 6 n doubles)
  int* pp = reinterpret_cast<int*>(c.red + SC_PIV);     // [2] pivot rows
  float* pinvb = reinterpret_cast<float*>(pp + 2);      // [2] pivot reciprocals
  float a[RS][CC];
#pragma unroll
  for (int s = 0; s < RS; ++s)
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      const int i = lane + 32 * s, j = wp + NW * cc;
      a[s][cc] = (i < n && j < n) ? A[i * ld + j] : 0.0f;
    }
  unsigned used = 0u;  // bit s: row lane + 32 s is a pivot row already
  // owner warp of column k: search, then publish the pivot and the column
  auto search = [&](int k, int buf) {
    const int ck = k / NW;
    float v[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) v[s] = 0.0f;
#pragma unroll
    for (int cc = 0; cc < CC; ++cc)
      if (cc == ck) {
#pragma unroll
        for (int s = 0; s < RS; ++s) v[s] = a[s][cc];
      }
    // argmax of |a_ik| over the unused rows, lowest row on ties, NaN never chosen: the
    // bit pattern of a non-negative float orders like its value, so key = bits + 1
    // (0: no candidate) goes through one warp max-reduction; the first row slot, then
    // the lowest lane, holding the maximum is the lowest row index that has it
    unsigned key[RS];
    unsigned kmax = 0u;
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      const int i = lane + 32 * s;
      const float x = fabsf(v[s]);
      key[s] = (i < n && !((used >> s) & 1u) && !isnan(x)) ? __float_as_uint(x) + 1u : 0u;
      kmax = max(kmax, key[s]);
    }
    const unsigned km = __reduce_max_sync(FULLMASK, kmax);
    int bi = n;
    float bval = 0.0f;
    if (km != 0u) {
#pragma unroll
      for (int s = 0; s < RS; ++s) {
        const unsigned b = __ballot_sync(FULLMASK, key[s] == km);
        if (bi == n && b != 0u) {
          const int l = __ffs(b) - 1;
          bi = l + 32 * s;
          bval = __shfl_sync(FULLMASK, v[s], l);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < RS; ++s)
      if (lane + 32 * s < n) pcol[buf * n + lane + 32 * s] = v[s];
    if (lane == 0) {
      const bool ok = bi < n && bval != 0.0f && isfinite(bval);
      pp[buf] = bi < n ? bi : k;  // no candidate (NaN column): a safe index, zero pivot
      pinvb[buf] = ok ? 1.0f / bval : 0.0f;
    }
  };
  if (wp == 0) search(0, 0);
  __syncthreads();
  int info = 0;
  for (int k = 0; k < n; ++k) {
    const int buf = k & 1;
    const int p = pp[buf];
    const float pinv = pinvb[buf];
    if (pinv == 0.0f && info == 0) info = k + 1;
    if (c.tid == 0) c.piv[k] = p;
    const int ps = p >> 5, pl = p & 31;
    float f[RS];
    bool isp[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      isp[s] = lane + 32 * s == p;
      f[s] = lane + 32 * s < n ? pcol[buf * n + lane + 32 * s] : 0.0f;
    }
    // column k becomes e_p (it then receives column k of the inverse)
    if (wp == k % NW) {
      const int ck = k / NW;
#pragma unroll
      for (int cc = 0; cc < CC; ++cc)
        if (cc == ck) {
#pragma unroll
          for (int s = 0; s < RS; ++s) a[s][cc] = isp[s] ? 1.0f : 0.0f;
        }
    }
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      float src = a[0][cc];
#pragma unroll
      for (int s = 1; s < RS; ++s) src = ps == s ? a[s][cc] : src;
      const float pr = __shfl_sync(FULLMASK, src, pl) * pinv;  // normalised pivot row
#pragma unroll
      for (int s = 0; s < RS; ++s) a[s][cc] = isp[s] ? pr : fmaf(-f[s], pr, a[s][cc]);
    }
#pragma unroll
    for (int s = 0; s < RS; ++s)
      if (isp[s]) used |= 1u << s;
    const int k1 = k + 1;
    if (k1 < n && wp == k1 % NW) search(k1, k1 & 1);
    __syncthreads();
  }
  // inverse permutation of the pivot rows, then the scatter into the true inverse
  for (int k = c.tid; k < n; k += NW * 32) c.perm[c.piv[k]] = k;
  __syncthreads();
#pragma unroll
  for (int s = 0; s < RS; ++s)
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
      const int i = lane + 32 * s, j = wp + NW * cc;
      if (i < n && j < n) A[c.perm[i] * ld + c.piv[j]] = a[s][cc];
    }
  __syncthreads();
  return info;
}

// Solve M x = b for the FP64 right-hand side b; x written as double.
// FP64: LU forward/back substitution. Otherwise: x = M32^-1 b with the FP32
// inverse, then `ir` sweeps of r = b - M0 x (FP64, against the assembled matrix
// M0) and x += M32^-1 r. One thread per row in every matrix-vector product.
template <int NW, int PREC>
__device__ void solve(Cta<NW>& c, int n, const double* b, double* x, int ir) {
  constexpr int NT = NW * 32;
  using P = Policy<PREC>;
  if constexpr (!P::IR) {
    for (int i = c.tid; i < n; i += NT) x[i] = b[c.perm[i]];
    __syncthreads();
    if (c.warp == Cta<NW>::SW) lu_solve_warp<double>(reinterpret_cast<double*>(c.M), n, c.invd, x, c.lane);
    __syncthreads();
  } else {
    using A = typename P::ASM;
    const float* Ai = reinterpret_cast<const float*>(c.M);
    const A* M0 = reinterpret_cast<const A*>(c.M0);
    float* xf = reinterpret_cast<float*>(c.sc);  // scratch vector reused as float
    ff2* xq = reinterpret_cast<ff2*>(c.rr);      // x as float-float pairs (rr is free in the solves)
    const int ld = odd_ld(n);
    for (int i = c.tid; i < n; i += NT) xf[i] = ff_split(b[i]).hi;
    __syncthreads();
    for (int i = c.tid; i < n; i += NT) {
      float acc = 0.0f;
      const float* row = Ai + i * ld;
      for (int j = 0; j < n; ++j) acc = fmaf(row[j], xf[j], acc);
      x[i] = f32_to_f64(acc);
      xq[i] = {acc, 0.0f};
    }
    __syncthreads();
    for (int sweep = 0; sweep < ir; ++sweep) {
      // Residual rows r = b - M0 x from the last warp down (the first warps carry the
      // species loops), as a compensated dot product on the FP32 pipe (Ogita, Rump and
      // Oishi's Dot2: exact products of the hi parts, TwoSum of the running sum, the
      // rounding errors and cross terms gathered in a second accumulator): as accurate as
      // a sum in about 48-bit arithmetic, then rounded to FP32 for the correction solve.
      for (int i = NT - 1 - c.tid; i < n; i += NT) {
        const ff2 bi = ff_split(b[i]);
        float sh = bi.hi, sl = bi.lo;
        const A* row = M0 + i * ld;
        for (int j = 0; j < n; ++j) {
          const ff2 xj = xq[j];
          float mh, ml = 0.0f;
          if constexpr (std::is_same<A, ff2>::value) {
            const ff2 mj = row[j];
            mh = mj.hi;
            ml = mj.lo;
          } else {
            mh = row[j];
          }
          const float p = __fmul_rn(mh, xj.hi);
          float pe = fmaf(mh, xj.hi, -p);
          pe = fmaf(mh, xj.lo, pe);
          if constexpr (std::is_same<A, ff2>::value) pe = fmaf(ml, xj.hi, pe);
          const ff2 t = two_sum(sh, -p);
          sh = t.hi;
          sl = __fadd_rn(sl, __fsub_rn(t.lo, pe));
        }
        xf[i] = __fadd_rn(sh, sl);
      }
      __syncthreads();
      for (int i = c.tid; i < n; i += NT) {
        float acc = 0.0f;
        const float* row = Ai + i * ld;
        for (int j = 0; j < n; ++j) acc = fmaf(row[j], xf[j], acc);
        x[i] += f32_to_f64(acc);
        if (sweep + 1 < ir) xq[i] = ff_split(x[i]);
      }
      __syncthreads();
    }
  }
}

// Factorisation of the iteration matrix: LU (FP64 form) or the FP32 inverse.
template <int NW, int PREC>
__device__ int factor(Cta<NW>& c, int n, bool pivot = true) {
  if constexpr (!Policy<PREC>::IR) {
    return lu_factor<NW, double>(c, reinterpret_cast<double*>(c.M), n, pivot);
  } else {
    float* A = reinterpret_cast<float*>(c.M);
    if constexpr (NW == 4) {
      if (n <= 56) return gj_invert_wc<4, 2, 14>(c, A, n);
      if (n <= 64) return gj_invert_wc<4, 2, 16>(c, A, n);
    } else if constexpr (NW == 8) {
      if (n <= 64) return gj_invert_wc<8, 2, 8>(c, A, n);
      if (n <= 128) return gj_invert_wc<8, 4, 16>(c, A, n);
    } else if constexpr (NW == 2) {
      if (n <= 64) return gj_invert_wc<2, 2, 32>(c, A, n);
    }
    return gj_invert<NW>(c, A, n);
  }
}

// Assemble the iteration matrix (fac = 1/(h gamma)) or the Jacobian (JO) in the
// policy's assembly precision, then give the LU its own copy when they differ.
template <int NW, int PREC, bool JO>
__device__ void build_matrix(const DevMech& m, Cta<NW>& c, const Scal& s, const double* f, double fac) {
  using P = Policy<PREC>;
  if constexpr (!P::IR) {
    assemble<NW, double, JO>(m, c, s, f, fac, c.M);
  } else {
    if constexpr (std::is_same<typename P::ASM, ff2>::value)
      assemble_ff<NW, JO>(m, c, s, f, fac, reinterpret_cast<ff2*>(c.M0));
    else
      assemble<NW, typename P::ASM, JO, true>(m, c, s, f, fac, c.M0);
    if (JO) return;
    const int n = m.K + 1, ld = odd_ld(n);
    const typename P::ASM* src = reinterpret_cast<const typename P::ASM*>(c.M0);
    float* dst = reinterpret_cast<float*>(c.M);
    for (int i = c.warp; i < n; i += NW)
      for (int j = c.lane; j < n; j += 32) dst[i * ld + j] = to_float(src[i * ld + j]);
    __syncthreads();
  }
}

// Iteration matrix (FP64 form) from a forward-difference Jacobian, column by column:
// J_.j = (f(y + d_j e_j) - f(y)) / d_j with d_j = sqrt(eps) max(|y_j|, floor_j)
// (floor 1 K for T, 1e-6 for mass fractions: a smaller floor lets rounding in f
// dominate the columns of trace species); S = sg J + fac I as in assemble.
// Costs n RHS evaluations: the classical alternative to the analytical Jacobian.
template <int NW, bool JO>
__device__ void fd_matrix(const DevMech& m, Cta<NW>& c, double p, const double* y, const double* f0, double fac) {
  constexpr int NT = NW * 32;
  const int n = m.K + 1, ld = odd_ld(n);
  double* A = reinterpret_cast<double*>(c.M);
  for (int j = 0; j < n; ++j) {
    const double d = 1.4901161193847656e-8 * fmax(fabs(y[j]), j == 0 ? 1.0 : 1e-6);
    for (int i = c.tid; i < n; i += NT) c.ys[i] = y[i] + (i == j ? d : 0.0);
    __syncthreads();
    eval_rhs<NW, false, false>(m, c, c.ys, p, c.fv);
    const double id = 1.0 / d;
    for (int i = c.tid; i < n; i += NT) {
      const double J = (c.fv[i] - f0[i]) * id;
      A[i * ld + j] = JO ? J : -J + (i == j ? fac : 0.0);
    }
    __syncthreads();
  }
}

// WRMS norm of e with scale atol + rtol max(|ya|, |yb|). With step_fac, also the
// step-size factor 0.9 err^(-1/q) (q = 4: RODAS4, 3: ROS34PW2; kFacMax for err = 0);
// both come from the CTA's last warp.
template <int NW>
__device__ double wrms(Cta<NW>& c, int n, const double* e, const double* ya, const double* yb,
                       double rtol, double atol, double* step_fac = nullptr, int q = 4) {
  constexpr int NT = NW * 32;
  double part[1] = {0.0};
  for (int i = c.tid; i < n; i += NT) {
    const double sc = atol + rtol * fmax(fabs(ya[i]), fabs(yb[i]));
    const double r = e[i] / sc;
    part[0] += r * r;
  }
  double o[2];
  c.reduce(part, warps_for<NW>(n), [&](const double (&t)[1], double (&r)[2]) {
    const double err = sqrt(t[0] / n);
    r[0] = err;
    r[1] = err > 0.0 ? kSafety / (q == 4 ? sqrt(sqrt(err)) : cbrt(err)) : kFacMax;
  }, o);
  if (step_fac) *step_fac = o[1];
  return o[0];
}

// Hairer-Wanner starting step (Solving ODEs I, Sec. II.4) in the WRMS norm with
// scale atol + rtol |y0|, exponent 1/q (the method's embedded order + 1), clamped
// to dt; a vanishing derivative selects the whole interval. Uses f0 = f(y0)
// (already in c.f0) and c.ys, c.fv.
template <int NW, bool FF = false>
__device__ double starting_step(const DevMech& m, Cta<NW>& c, double p, double dt, double rtol,
                                double atol, int q = 4) {
  constexpr int NT = NW * 32;
  const int n = m.K + 1;
  const double d0 = wrms(c, n, c.y, c.y, c.y, rtol, atol);
  const double d1 = wrms(c, n, c.f0, c.y, c.y, rtol, atol);
  double ha = (d1 > 1e-300) ? 0.01 * d0 / d1 : dt;
  ha = fmin(ha, dt);
  for (int i = c.tid; i < n; i += NT) c.ys[i] = c.y[i] + ha * c.f0[i];
  __syncthreads();
  eval_rhs<NW, false, FF>(m, c, c.ys, p, c.fv);
  for (int i = c.tid; i < n; i += NT) c.rr[i] = c.fv[i] - c.f0[i];
  __syncthreads();
  const double d2 = wrms(c, n, c.rr, c.y, c.y, rtol, atol) / ha;
  const double mx = fmax(d1, d2);
  const double hb = (mx > 1e-300) ? (q == 4 ? pow(0.01 / mx, 0.25) : cbrt(0.01 / mx)) : dt;
  return fmin(fmin(100.0 * ha, hb), dt);
}

// Mass enthalpy and heat capacity at T for mass fractions Y (CTA sums).
template <int NW>
__device__ void h_cp_mass(const DevMech& m, Cta<NW>& c, double T, const double* Y, double& h,
                          double& cp) {
  constexpr int NT = NW * 32;
  const double invT = 1.0 / T;
  double part[2] = {0.0, 0.0};
  for (int k = c.tid; k < m.K; k += NT) {
    const double* a = m.nasa + 36 * k;
    a += (T < a[34]) ? 0 : 17;
    const double cpr = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double hr = a[5] + T * (a[6] + T * (a[7] + T * (a[8] + T * a[9]))) + a[10] * invT;
    part[0] += Y[k] * hr * m.invW[k];
    part[1] += Y[k] * cpr * m.invW[k];
  }
  c.sum(part, warps_for<NW>(m.K));
  h = part[0] * kRc * T;
  cp = part[1] * kRc;
}

// ---------------------------------------------------------------------------
// one cell
// ---------------------------------------------------------------------------
// Per-phase cycle counters (diagnostic; thread 0 reads the clock right after the
// CTA barriers that close each phase): 0 load + starting step, 1 RHS and Jacobian
// data at the step point, 2 iteration-matrix assembly, 3 factorisation, 4 stage RHS,
// 5 stage solves, 6 stage combination + error norm + control, 7 T recovery + store.
#define PHASE(k)                                                              \
  do {                                                                        \
    if (prof) {                                                               \
      const long long now_ = clock64();                                       \
      atomicAdd(args.phase + cur_, (unsigned long long)(now_ - last_));       \
      last_ = now_;                                                           \
      cur_ = (k);                                                             \
    }                                                                         \
  } while (0)

template <int NW, int PREC, int MTH>
__device__ void integrate_cell(const Job& job, int64_t cell, const IntegrateArgs& args, Cta<NW>& c) {
  using MT = Meth<MTH>;
  const bool prof = args.phase != nullptr && c.tid == 0;
  long long last_ = prof ? clock64() : 0;
  int cur_ = 0;
  constexpr int NT = NW * 32;
  const DevMech& m = job.m;
  const int K = m.K, n = K + 1;
  const double p = job.p[cell];
  const double dt = args.dt, rtol = args.rtol, atol = args.atol;
  // load (coalesced over species)
  if (c.tid == 0) c.y[0] = job.T[cell];
  for (int k = c.tid; k < K; k += NT) c.y[1 + k] = job.Y[(size_t)cell * K + k];
  __syncthreads();
  int status = CHEM_CELL_OK;
  {
    double part[1] = {0.0};
    for (int i = c.tid; i < n; i += NT) part[0] += isfinite(c.y[i]) ? 0.0 : 1.0;
    c.sum(part, warps_for<NW>(n));
    if (part[0] > 0.0 || !(c.y[0] > 0.0) || !(p > 0.0)) status = CHEM_CELL_NONFINITE;
  }
  int steps = 0, rejects = 0;
  double h_first = 0.0, h_next = 0.0;
  if (status == CHEM_CELL_OK) {
    double h_target, cp_dummy;
    h_cp_mass(m, c, c.y[0], c.y + 1, h_target, cp_dummy);
    // initial step
    double h = -1.0;
    bool guard = false;  // a supplied initial step, checked against f(y0) at the first step
    if (args.use_h0 && job.h0) {
      const double g = job.h0[cell];
      if (isfinite(g) && g > 0.0) {
        h = fmin(g, dt);
        guard = args.h0_guard != 0;
      }
    }
    if (h <= 0.0) {
      eval_rhs<NW, false, Policy<PREC>::IR>(m, c, c.y, p, c.f0);
      h = starting_step<NW, Policy<PREC>::IR>(m, c, p, dt, rtol, atol, MT::Q);
    }
    double t = 0.0, h_unclipped = h;
    bool after_reject = false;
    while (true) {
      if (dt - t <= 1e-12 * dt) break;
      if (steps >= args.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
      if (!(h >= kHmin)) { status = CHEM_CELL_H_UNDERFLOW; break; }  // also catches NaN
      h_unclipped = h;
      if (t + h > dt) h = dt - t;
      ++steps;
      // Jacobian and f0 at y; iteration matrix; factorisation
      PHASE(1);
      // A supplied initial step (learned or carried over) is kept inside the starting
      // step heuristic's envelope [h_a, 100 h_a], h_a = 0.01 |y0| / |f(y0)| in the WRMS
      // norm: f(y0) is the first step's first-stage RHS, so the check costs no RHS
      // evaluation, and a prediction far from the states it was trained on cannot cost
      // more than the heuristic's own range of answers.
      auto apply_guard = [&]() {
        if (!guard) return;
        guard = false;
        const double d0 = wrms(c, n, c.y, c.y, c.y, rtol, atol);
        const double d1 = wrms(c, n, c.f0, c.y, c.y, rtol, atol);
        const double ha = d1 > 1e-300 ? 0.01 * d0 / d1 : dt;
        h = fmin(fmin(fmax(h, ha), 100.0 * ha), dt - t);
        h_unclipped = h;
      };
      if (PREC == PREC_FP64 && args.jac_fd) {
        eval_rhs<NW, false, false>(m, c, c.y, p, c.f0);
        apply_guard();
        PHASE(2);
        fd_matrix<NW, false>(m, c, p, c.y, c.f0, 1.0 / (h * MT::gamma(args)));
      } else {
        const Scal s = eval_rhs<NW, true, Policy<PREC>::IR>(m, c, c.y, p, c.f0);
        apply_guard();
        PHASE(2);
        build_matrix<NW, PREC, false>(m, c, s, c.f0, 1.0 / (h * MT::gamma(args)));
      }
      PHASE(3);
      const int info = factor<NW, PREC>(c, n, !(PREC == PREC_FP64 && args.no_pivot));
      PHASE(6);
      double err, step_fac = kFacMin;
      if (info != 0) {
        err = NAN;
      } else {
        const double invh = 1.0 / h;
        constexpr int S = MT::S;
#pragma unroll 1
        for (int st = 0; st < S; ++st) {
          const double* fs = c.f0;
          if (st > 0) {
            PHASE(6);
            for (int i = c.tid; i < n; i += NT) {
              double v = c.y[i];
              for (int j = 0; j < st; ++j) v += MT::a(args, st, j) * c.u[j * n + i];
              c.ys[i] = v;
            }
            __syncthreads();
            PHASE(4);
            eval_rhs<NW, false, Policy<PREC>::IR>(m, c, c.ys, p, c.fv);
            fs = c.fv;
          }
          PHASE(6);
          // stage right-hand side f(y_s) + sum_j (c_sj / h) u_j, in place in fv
          for (int i = c.tid; i < n; i += NT) {
            double v = 0.0;
            for (int j = 0; j < st; ++j) v += MT::c(args, st, j) * c.u[j * n + i];
            c.fv[i] = fma(invh, v, fs[i]);
          }
          __syncthreads();
          PHASE(5);
          solve<NW, PREC>(c, n, c.fv, c.u + st * n, args.ir_sweeps);
        }
        PHASE(6);
        for (int i = c.tid; i < n; i += NT) {
          double v = c.y[i], e = 0.0;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            v += MT::m(args, j) * c.u[j * n + i];
            if (!MT::E_LAST) e += MT::e(args, j) * c.u[j * n + i];
          }
          c.yn[i] = v;
          if (!MT::E_LAST) c.rr[i] = e;
        }
        __syncthreads();
        err = wrms(c, n, MT::E_LAST ? c.u + (S - 1) * n : c.rr, c.y, c.yn, rtol, atol, &step_fac, MT::Q);
      }
      if (!(err <= 1.0)) {
        ++rejects;
        after_reject = true;
        h *= isfinite(err) ? fmax(step_fac, kFacMin) : kFacMin;
        continue;
      }
      t += h;
      for (int i = c.tid; i < n; i += NT) c.y[i] = c.yn[i];
      __syncthreads();
      if (h_first == 0.0) h_first = h;
      const double fac = fmin(fmax(step_fac, kFacMin), after_reject ? 1.0 : kFacMax);
      after_reject = false;
      h *= fac;
    }
    // step size to carry to the next call: the controller's proposal, or the step
    // before the final clipping to dt when that was longer
    h_next = fmax(h, h_unclipped);
    // temperature from the conserved mass enthalpy (Newton, |dT| < 1e-10 T)
    PHASE(7);
    if (status == CHEM_CELL_OK) {
      double T = c.y[0];
      for (int it = 0; it < 50; ++it) {
        double hm, cpm;
        h_cp_mass(m, c, T, c.y + 1, hm, cpm);
        const double dT = (hm - h_target) / cpm;
        T -= dT;
        if (fabs(dT) < 1e-10 * T) break;
      }
      if (!(T >= kTmin && T <= kTmax)) status = CHEM_CELL_T_RANGE;
      else if (c.tid == 0) c.y[0] = T;
      __syncthreads();
    }
  }
  // store (the last accepted state for failed cells)
  if (status != CHEM_CELL_NONFINITE) {
    if (c.tid == 0) job.T[cell] = c.y[0];
    for (int k = c.tid; k < K; k += NT) job.Y[(size_t)cell * K + k] = c.y[1 + k];
  }
  PHASE(7);
  if (c.tid == 0) {
    if (job.st.substeps) job.st.substeps[cell] = steps;
    if (job.st.rejects) job.st.rejects[cell] = rejects;
    if (job.st.h_first) job.st.h_first[cell] = h_first;
    if (job.st.status) job.st.status[cell] = status;
    if (job.st.h_last) job.st.h_last[cell] = status == CHEM_CELL_OK ? h_next : 0.0;
    if (job.cost_out) job.cost_out[cell] = (float)steps;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Launch bounds: 128 registers a thread for four CTAs of 128 threads (FP64 form: its
// shared-memory footprint allows no more up to ~60 species), eight of 64 or two of 256;
// the mixed form with 128 threads takes 96 registers for five CTAs per SM, which its
// global-memory matrix slot makes room for (measured on 54 species: 7 % faster than
// four CTAs; six and seven CTAs spill too much in the register Gauss-Jordan).
template <int NW, int PREC, int MTH>
__global__ void __launch_bounds__(NW * 32, NW == 4 ? (PREC == PREC_MIXED ? 5 : 4) : NW == 2 ? 8 : 2) k_integrate(const __grid_constant__ IntegrateArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_work;
  const bool m0g = PREC == PREC_MIXED && args.m0_scratch != nullptr;
  const Layout L = make_layout(args.smem_K, args.smem_I, PREC, m0g);
  Cta<NW> c;
  c.bind(smem, L);
  if (m0g) c.M0 = args.m0_scratch + (size_t)blockIdx.x * args.m0_stride;
  for (long long it = 0;; ++it) {
    long long w;
    if (args.sched == SCHED_PLAIN) {
      if (it > 0) break;
      w = blockIdx.x;
    } else if (args.sched == SCHED_STATIC) {
      w = blockIdx.x + it * (long long)gridDim.x;
    } else {
      if (threadIdx.x == 0) s_work = atomicAdd(args.queue, 1);
      __syncthreads();
      w = s_work;
      __syncthreads();
    }
    if (w >= args.n_total) break;
    const long long g = args.perm ? args.perm[w] : w;
    int j = 0;
    while (j + 1 < args.n_jobs && g >= args.jobs[j + 1].offset) ++j;
    integrate_cell<NW, PREC, MTH>(args.jobs[j], g - args.jobs[j].offset, args, c);
  }
}

// ---------------------------------------------------------------------------
// launch helper
// ---------------------------------------------------------------------------
template <class KernelT>
static cudaError_t prep(KernelT k, size_t smem) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int NW, int PREC, int MTH>
static cudaError_t launch_integrate_m(const IntegrateArgs& a, int grid, cudaStream_t st) {
  const size_t smem = smem_bytes(a.smem_K, a.smem_I, PREC, a.m0_scratch != nullptr);
  cudaError_t e = prep(k_integrate<NW, PREC, MTH>, smem);
  if (e != cudaSuccess) return e;
  k_integrate<NW, PREC, MTH><<<grid, NW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chem
