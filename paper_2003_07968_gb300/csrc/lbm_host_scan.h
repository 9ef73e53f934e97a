// lbm_host_scan.h -- host-side scan of the fields handed to lbm_init and
// lbm_submit (host code only; no device code includes it).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <functional>
#include <thread>
#include <vector>

namespace pplbm {

// One pass over a host field: its smallest value into *mn, and whether every
// value is finite (x * 0 is 0 for a finite x and NaN otherwise, so the sum
// of those products stays 0 exactly when all are finite).  Four independent
// accumulators per thread keep the loop vectorisable; fields of a million
// values or more are split across up to 16 threads.
inline bool field_scan(const double* v, size_t n, double* mn) {
    auto scan = [v](size_t b, size_t e, double& m, double& z) {
        double m0 = HUGE_VAL, m1 = HUGE_VAL, m2 = HUGE_VAL, m3 = HUGE_VAL;
        double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0;
        size_t i = b;
        for (; i + 4 <= e; i += 4) {
            m0 = v[i] < m0 ? v[i] : m0;
            m1 = v[i + 1] < m1 ? v[i + 1] : m1;
            m2 = v[i + 2] < m2 ? v[i + 2] : m2;
            m3 = v[i + 3] < m3 ? v[i + 3] : m3;
            z0 += v[i] * 0.0;
            z1 += v[i + 1] * 0.0;
            z2 += v[i + 2] * 0.0;
            z3 += v[i + 3] * 0.0;
        }
        for (; i < e; ++i) {
            m0 = v[i] < m0 ? v[i] : m0;
            z0 += v[i] * 0.0;
        }
        m = std::min(std::min(m0, m1), std::min(m2, m3));
        z = (z0 + z1) + (z2 + z3);
    };
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = n < ((size_t)1 << 20) ? 1 : std::min<size_t>({hw, 16, n >> 18});
    std::vector<double> m(nt), z(nt);
    std::vector<std::thread> th;
    const size_t chunk = (n + nt - 1) / nt;
    size_t t = 1;
    // no exception may leave a C entry point: chunks without a thread (its
    // creation failed) are scanned on this thread
    try {
        for (; t < nt; ++t)
            th.emplace_back(scan, std::min(n, t * chunk), std::min(n, (t + 1) * chunk),
                            std::ref(m[t]), std::ref(z[t]));
    } catch (...) {
    }
    for (size_t u = t; u < nt; ++u) scan(std::min(n, u * chunk), std::min(n, (u + 1) * chunk), m[u], z[u]);
    scan(0, std::min(n, chunk), m[0], z[0]);
    for (auto& w : th) w.join();
    double mm = HUGE_VAL, zz = 0.0;
    for (size_t t = 0; t < nt; ++t) {
        mm = std::min(mm, m[t]);
        zz += z[t];
    }
    *mn = mm;
    return zz == 0.0;
}

}  // namespace pplbm
