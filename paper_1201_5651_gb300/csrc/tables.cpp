// Frequency-integrated photoionisation-rate tables (Mackey 2012, Sect. 2: the
// multi-frequency rates are precomputed for a source spectrum and tabulated
// against column; Sect. 4: blackbody sources).
//
// For a spectrum phi(nu) of photons per unit frequency and the cross-section
// sigma_nu = sigma0 (nu/nu0)^-3, the photon rate left after a neutral column N
// is P(N) = Q int phi e^{-sigma N} / int phi.  The table stores, at K
// log-spaced columns, ln(P/Q) and its first and second derivatives in ln N:
//   d ln P / d ln N = -N <sigma>,
//   d2 ln P / d(ln N)^2 = -N <sigma> + N^2 var(sigma),
// averages weighted by phi e^{-sigma N}.  The device interpolates ln P with
// the quintic Hermite polynomial through those values on every interval; this
// file hands it the monomial coefficients of each interval.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "tables.h"

namespace oots {

// Gauss-Legendre nodes and weights on [-1,1] by Newton iteration on P_n
// (initial guesses from the asymptotic cosine formula).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static HostTable make_table(int kind, double T, double sigma0, int K, double lnN_lo, double lnN_hi)
{
    HostTable H;
    H.K = K;
    H.lnN_lo = lnN_lo;
    H.lnN_hi = lnN_hi;
    H.dl = (lnN_hi - lnN_lo) / (K - 1);
    H.L.resize(K);
    H.D1.resize(K);
    H.D2.resize(K);
    if (kind == 0) {
        for (int k = 0; k < K; k++) {
            double N = std::exp(lnN_lo + k * H.dl);
            H.L[k] = H.D1[k] = H.D2[k] = -sigma0 * N;
        }
    } else {
        // quadrature nodes in x = nu/nu0 on [1, 40]: 512 log-spaced panels x 12 points
        const double theta = (13.6 / 8.617333262e-5) / T;   // h nu0 / k T, h nu0 = 13.6 eV
        const int npan = 512, ng = 12;
        std::vector<double> gx, gw;
        gauss_legendre(ng, gx, gw);
        std::vector<double> xs, lw, sg;   // node, ln(weight * phi), sigma
        xs.reserve(npan * ng);
        const double r = std::pow(40.0, 1.0 / npan);
        double a = 1.0;
        for (int p = 0; p < npan; p++) {
            double b = (p == npan - 1) ? 40.0 : a * r;
            for (int g = 0; g < ng; g++) {
                double xv = 0.5 * (a + b) + 0.5 * (b - a) * gx[g];
                double phi = xv * xv / std::expm1(theta * xv);
                xs.push_back(xv);
                lw.push_back(std::log(0.5 * (b - a) * gw[g] * phi));
                sg.push_back(sigma0 / (xv * xv * xv));
            }
            a = b;
        }
        const size_t M = xs.size();
        double lnZ;
        {
            double mx = -1e308;
            for (size_t q = 0; q < M; q++) mx = std::fmax(mx, lw[q]);
            double s = 0.0;
            for (size_t q = 0; q < M; q++) s += std::exp(lw[q] - mx);
            lnZ = mx + std::log(s);
        }
        for (int k = 0; k < K; k++) {
            double N = std::exp(lnN_lo + k * H.dl);
            double mx = -1e308;
            for (size_t q = 0; q < M; q++) mx = std::fmax(mx, lw[q] - sg[q] * N);
            double m0 = 0.0, m1 = 0.0;
            for (size_t q = 0; q < M; q++) {
                double e = std::exp(lw[q] - sg[q] * N - mx);
                m0 += e;
                m1 += e * sg[q];
            }
            double mu = m1 / m0, v = 0.0;
            for (size_t q = 0; q < M; q++) {
                double e = std::exp(lw[q] - sg[q] * N - mx);
                v += e * (sg[q] - mu) * (sg[q] - mu);
            }
            v /= m0;
            if (sigma0 * N < 0.1) {
                // thin columns: ln(P/Q) = log1p(sum w phi (e^{-sigma N} - 1) / Z) without cancellation
                double def = 0.0, Z = 0.0;
                for (size_t q = 0; q < M; q++) {
                    const double wq = std::exp(lw[q] - lnZ);
                    def += wq * std::expm1(-sg[q] * N);
                    Z += wq;
                }
                H.L[k] = std::log1p(def / Z);
            } else {
                H.L[k] = mx + std::log(m0) - lnZ;
            }
            H.D1[k] = -N * mu;
            H.D2[k] = -N * mu + N * N * v;
        }
    }
    // monomial coefficients of the quintic Hermite interpolant in t = (lnN - lnN_k)/dl
    H.coef.resize(6 * (K - 1));
    for (int k = 0; k + 1 < K; k++) {
        double y0 = H.L[k], y1 = H.L[k + 1];
        double p0 = H.D1[k] * H.dl, p1 = H.D1[k + 1] * H.dl;
        double q0 = H.D2[k] * H.dl * H.dl, q1 = H.D2[k + 1] * H.dl * H.dl;
        double d = y1 - y0;
        double *c = &H.coef[6 * k];
        c[0] = y0;
        c[1] = p0;
        c[2] = 0.5 * q0;
        c[3] = 10.0 * d - 6.0 * p0 - 4.0 * p1 - 1.5 * q0 + 0.5 * q1;
        c[4] = -15.0 * d + 8.0 * p0 + 7.0 * p1 + 1.5 * q0 - q1;
        c[5] = 6.0 * d - 3.0 * p0 - 3.0 * p1 - 0.5 * q0 + 0.5 * q1;
    }
    H.Nnode.resize(K);
    for (int k = 0; k < K; k++) H.Nnode[k] = std::exp(lnN_lo + k * H.dl);
    H.a0 = -std::expm1(H.L[0]);
    return H;
}

const HostTable &host_table(int kind, double T, double sigma0)
{
    static std::mutex mu;
    static std::map<std::pair<int, std::pair<double, double>>, HostTable> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(kind, std::make_pair(kind == 0 ? 0.0 : T, sigma0));
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    HostTable H = make_table(kind, T, sigma0, TABLE_K, TABLE_LNN_LO, TABLE_LNN_HI);
    return cache.emplace(key, std::move(H)).first->second;
}

} // namespace oots
