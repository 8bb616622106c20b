// Host-side FCF construction (Sec. 3.2, Algorithms 1-2); see fcf.cpp.
#pragma once

#include <complex>
#include <vector>

namespace rexi {

struct dd;
double sqrt_t(double x);
dd sqrt_t(dd x);

struct FcfResult {
    int K = 0;
    double R1 = 0.0;
    int L = 0;
    double sigma_K1 = 0.0;       // sigma_{K+1} of Theorem 1
    double min_re_sigma = 0.0;   // min_k |Re sigma_k|: distance of the poles from i[-R1,R1]
    double amplification = 0.0;  // max_{w in i[-R1,R1]} sum |beta_k| / |w - sigma_k|
    std::vector<std::complex<double>> sigma, beta, z;
};

// 0 on success, -1 bad argument, -6 construction failure (see rexi.h REXI_EPLAN).
int fcf_construct(int K, double R1, FcfResult* out);
int fcf_cached(int K, double R1, FcfResult* out);
// Largest R1 (floored to an integer when >= 2) with 2 sigma_{K+1}(R1) <= eps_target.
double fcf_default_R1(int K, double eps_target);
double fcf_default_R1_cached(int K, double eps_target);
// J_0(R) .. J_L(R) (Miller's backward recurrence in double-double, rounded).
std::vector<double> bessel_j(int L, double R);

}  // namespace rexi
