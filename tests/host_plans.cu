// Host-side dump of the row stage's FFT plans, twiddle-table layout, table
// pitch and the pivot recurrence's fixed point, for tests/test_host_plans.py
// (compiled for the host only; no GPU call).
#include <cstdio>

#include "../paper_1507_05988_gb300/csrc/fcn_device.cuh"

using namespace fcn;

int main() {
    for (int nt = 2; nt <= 8192; nt *= 2) {
        for (int plan = 0; plan < 2; ++plan) {
            const int ntp = fft_tag(nt, plan);
            std::printf("plan %d %d %d %d %d", nt, plan, fft_npass(ntp), tw_size(ntp), table_pitch(nt));
            for (int p = 0; p < fft_npass(ntp); ++p) std::printf(" %d:%d:%d", fft_radix(ntp, p), fft_ns(ntp, p), tw_offset(ntp, p));
            std::printf("\n");
        }
    }
    const double ss[] = {0.0, 7e-3, 0.66, 3.0, 40.0};
    const double dks[] = {0.0, 6e-7, 1e-3};
    const int qs[] = {0, 1, 17, 2048};
    for (double s : ss)
        for (double dk : dks)
            for (int q : qs) {
                const cx<double> v = piv_limit(s, dk, q);
                std::printf("lim %.17g %.17g %d %.17g %.17g\n", s, dk, q, v.x, v.y);
            }
    return 0;
}
