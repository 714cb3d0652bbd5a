// Host-side check of the row stage's chunked time-domain row I/O (RowIo,
// row_chunks; RowIoReal, row_real_chunks for the rho output) for
// tests/test_host_plans.py: for every Nt, FFT plan and
// precision where it applies, the threads' chunks cover the row exactly once,
// every value lands at its digit-reversed position, and the shared-memory
// wavefronts per warp instruction are counted against the per-value loop it
// replaces.  Compiled for the host only; no GPU call.
#include <cstdio>
#include <vector>

#include "../paper_1507_05988_gb300/csrc/row_kernel.cuh"

using namespace fcn;

// Wavefronts of one warp access to S: 32 banks of 4 bytes; lanes touching
// different words of one bank are serialised.
static int wavefronts(const std::vector<long> &byte_addr, int bytes) {
    std::vector<std::vector<long>> words(32);
    for (long a : byte_addr)
        for (int k = 0; k < bytes / 4; ++k) {
            const long wd = a / 4 + k;
            auto &v = words[wd % 32];
            bool seen = false;
            for (long x : v) seen = seen || x == wd;
            if (!seen) v.push_back(wd);
        }
    size_t m = 0;
    for (auto &v : words) m = v.size() > m ? v.size() : m;
    return (int)m;
}

template <typename T, int NT>
static int check() {
    using C = RowCfg<NT>;
    using IO = RowIo<T, NT>;
    const int N = fft_nt(NT);
    const int plan = fft_plan(NT);
    if (!IO::OK) {
        std::printf("io %s %d %d skip\n", sizeof(T) == 4 ? "f32" : "f64", N, plan);
        return 0;
    }
    std::vector<int> hits(N, 0);
    int bad = 0;
    // chunk visits of every thread, in order (the k-th call is the k-th instruction)
    std::vector<std::vector<int>> taus(C::TPR), pos(C::TPR);
    for (int t = 0; t < C::TPR; ++t)
        row_chunks<T, NT>(t, [&](int tau, int q0, int p0) {
            if (tau % IO::CPC != 0 || tau < 0 || tau + IO::CPC > N) { ++bad; return; }
            for (int m = 0; m < IO::CPC; ++m) {
                const int q = own_idx<NT, IO::NSL>(q0, p0, (tau & 15) + m);
                if (q != pidx(tpos<NT>(tau + m), N) || q < 0 || q >= C::PADN) ++bad;
                ++hits[tau + m];
                taus[t].push_back(tau + m);
                pos[t].push_back(q);
            }
        });
    for (int i = 0; i < N; ++i) bad += hits[i] != 1;
    // shared-memory wavefronts per warp instruction: new (chunk) order
    // against the per-value loop (lane t moves tau = t + TPR i)
    int wf_new = 0, wf_old = 0, sectors_new = 0;
    for (int w = 0; w < C::TPR / 32; ++w) {
        for (size_t k = 0; k < taus[32 * w].size(); ++k) {
            std::vector<long> a;
            std::vector<long> sec;
            for (int l = 0; l < 32; ++l) {
                a.push_back((long)pos[32 * w + l][k] * (long)sizeof(cx<T>));
                const long s = (long)taus[32 * w + l][k] * (long)sizeof(cx<T>) / 32;
                bool seen = false;
                for (long x : sec) seen = seen || x == s;
                if (!seen) sec.push_back(s);
            }
            const int f = wavefronts(a, sizeof(cx<T>));
            wf_new = f > wf_new ? f : wf_new;
            sectors_new = (int)sec.size() > sectors_new ? (int)sec.size() : sectors_new;
        }
        for (int i = 0; i < C::E; ++i) {
            std::vector<long> a;
            for (int l = 0; l < 32; ++l) a.push_back((long)pidx(tpos<NT>(32 * w + l + C::TPR * i), N) * (long)sizeof(cx<T>));
            const int f = wavefronts(a, sizeof(cx<T>));
            wf_old = f > wf_old ? f : wf_old;
        }
    }
    std::printf("io %s %d %d bad %d wf_new %d wf_old %d sectors %d\n", sizeof(T) == 4 ? "f32" : "f64", N, plan, bad,
                wf_new, wf_old, sectors_new);
    return bad;
}

// The rho output's chunks of reals, read from the u rows (T per value).
template <typename T, int NT>
static int check_real() {
    using C = RowCfg<NT>;
    using IO = RowIoReal<T, NT>;
    const int N = fft_nt(NT);
    const int plan = fft_plan(NT);
    if (!IO::OK) {
        std::printf("rio %s %d %d skip\n", sizeof(T) == 4 ? "f32" : "f64", N, plan);
        return 0;
    }
    std::vector<int> hits(N, 0);
    int bad = 0;
    std::vector<std::vector<int>> taus(C::TPR), pos(C::TPR);
    for (int t = 0; t < C::TPR; ++t)
        row_real_chunks<T, NT>(t, [&](int tau) {
            if (tau % IO::RC != 0 || tau < 0 || tau + IO::RC > N || (tau & ~15) != ((tau + IO::RC - 1) & ~15)) {
                ++bad;
                return;
            }
            const int p0 = tpos<NT>(tau & ~15);
            const int q0 = pidx(p0, N);
            for (int m = 0; m < IO::RC; ++m) {
                const int q = own_idx<NT, PassCfg<NT, C::NPASS - 1>::NS>(q0, p0, (tau & 15) + m);
                if (q != pidx(tpos<NT>(tau + m), N) || q < 0 || q >= C::PADN) ++bad;
                ++hits[tau + m];
                taus[t].push_back(tau + m);
                pos[t].push_back(q);
            }
        });
    for (int i = 0; i < N; ++i) bad += hits[i] != 1;
    int wf_new = 0, wf_old = 0;
    for (int w = 0; w < C::TPR / 32; ++w) {
        for (size_t k = 0; k < taus[32 * w].size(); ++k) {
            std::vector<long> a;
            for (int l = 0; l < 32; ++l) a.push_back((long)pos[32 * w + l][k] * (long)sizeof(T));
            const int f = wavefronts(a, sizeof(T));
            wf_new = f > wf_new ? f : wf_new;
        }
        for (int i = 0; i < C::E; ++i) {
            std::vector<long> a;
            for (int l = 0; l < 32; ++l) a.push_back((long)pidx(tpos<NT>(32 * w + l + C::TPR * i), N) * (long)sizeof(T));
            const int f = wavefronts(a, sizeof(T));
            wf_old = f > wf_old ? f : wf_old;
        }
    }
    std::printf("rio %s %d %d bad %d wf_new %d wf_old %d\n", sizeof(T) == 4 ? "f32" : "f64", N, plan, bad, wf_new,
                wf_old);
    return bad;
}

template <typename T, int NT>
static int both() {
    return check<T, NT>() + check<T, fft_tag(NT, 1)>() + check_real<T, NT>() + check_real<T, fft_tag(NT, 1)>();
}

template <typename T>
static int all_nt() {
    return both<T, 16>() + both<T, 32>() + both<T, 64>() + both<T, 128>() + both<T, 256>() + both<T, 512>() +
           both<T, 1024>() + both<T, 2048>() + both<T, 4096>() + both<T, 8192>();
}

int main() {
    const int bad = all_nt<float>() + all_nt<double>();
    std::printf("total_bad %d\n", bad);
    return bad ? 1 : 0;
}
