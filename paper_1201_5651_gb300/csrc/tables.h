// Host-side rate tables (built in FP64 at set-up, uploaded to the device).
#pragma once
#include <vector>

namespace oots {

// 512 nodes, log10 N from 10 to 24 [cm^-2]
constexpr int TABLE_K = 512;
constexpr double TABLE_LNN_LO = 10.0 * 2.302585092994045684;
constexpr double TABLE_LNN_HI = 24.0 * 2.302585092994045684;

struct HostTable {
    int K;
    double lnN_lo, lnN_hi, dl;
    std::vector<double> L, D1, D2;   // ln(P/Q) and its first two ln N derivatives at the nodes
    std::vector<double> coef;        // (K-1) x 6 monomial coefficients per interval
    std::vector<double> Nnode;       // node columns
    double a0;                       // 1 - P(N0)/Q
};

// kind 0: all photons at nu0 (exact exponential); kind 1: blackbody at T.
// Cached per (kind, T, sigma0); thread-safe.
const HostTable &host_table(int kind, double T, double sigma0);

} // namespace oots
