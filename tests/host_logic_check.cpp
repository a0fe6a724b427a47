// Host checks of two pieces of the library's pure host logic, compiled against its own
// headers:
//   * split_units (segments.h): how serving's large lane cuts a solve's ordered product
//     work into launches -- contiguous, covering, non-empty parts, at most the part
//     limit, each within one unit of the even share;
//   * tuning_to_json / tuning_from_json (tuning_json.h): the autotune cache as JSON --
//     every written cache reads back identically, and malformed, foreign or
//     out-of-range text is rejected without changing the output;
//   * Arena (arena.h): the serving loop's first-fit placement of request workspaces --
//     against a brute-force model of the free ranges, under random alloc / release
//     sequences: live ranges never overlap and stay inside the arena, each alloc takes
//     the lowest free range that fits and fails only when none does, free ranges stay
//     disjoint and coalesced, and releasing everything restores one range.
//
// Usage: host_logic_check <seed>; prints "<n> failures" and exits 0 when there are none.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <iterator>
#include <map>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "arena.h"
#include "segments.h"
#include "tuning_json.h"

namespace {

int failures = 0;

void expect(bool ok, const char *what, long long a = 0, long long b = 0)
{
    if (!ok) {
        ++failures;
        if (failures <= 20)
            std::printf("FAIL %s (%lld, %lld)\n", what, a, b);
    }
}

void check_split(std::mt19937_64 &rng)
{
    // fixed cases
    expect(svt::split_units({}, 1.0, 8) == std::vector<int>{0, 0}, "empty list");
    expect(svt::split_units({5.0}, 1.0, 8) == std::vector<int>{0, 1}, "one unit");
    expect(svt::split_units({1, 1, 1, 1}, 1e9, 8) == std::vector<int>{0, 4}, "one part");
    expect(svt::split_units({1, 1, 1, 1}, 1.0, 8) == std::vector<int>{0, 1, 2, 3, 4}, "one per unit");
    expect(svt::split_units({1, 1, 1, 1, 1, 1}, 1.0, 3) == std::vector<int>{0, 2, 4, 6}, "part limit");
    expect(svt::split_units({0, 0, 0}, 1.0, 8) == std::vector<int>{0, 3}, "zero work");
    // random lists
    std::uniform_int_distribution<int> len(1, 300), lim(1, 64);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    for (int trial = 0; trial < 3000; ++trial) {
        const int n = len(rng), max_parts = lim(rng);
        std::vector<double> w(n);
        double total = 0.0, wmax = 0.0;
        for (double &x : w) {
            const double r = u(rng);
            x = r < 0.1 ? 0.0 : (r < 0.2 ? 50.0 * u(rng) : u(rng));  // zeros, a few large units
            total += x;
            wmax = std::max(wmax, x);
        }
        const double target = total * std::exp(std::log(1e-3) + u(rng) * std::log(1e4));
        const std::vector<int> b = svt::split_units(w, target, max_parts);
        const int parts = (int)b.size() - 1;
        const int want = (int)std::min<double>(max_parts, std::max(1.0, std::ceil(total / std::max(target, 1.0))));
        expect(b.front() == 0 && b.back() == n, "covers the list", b.front(), b.back());
        expect(parts >= 1 && parts <= std::min(want, n), "part count", parts, want);
        const double per = total / want;
        for (int k = 0; k < parts; ++k) {
            expect(b[k + 1] > b[k], "non-empty part", b[k], b[k + 1]);
            double pw = 0.0;
            for (int i = b[k]; i < b[k + 1]; ++i)
                pw += w[i];
            expect(pw <= per + wmax + 1e-9 * total, "part within one unit of the share", k, parts);
        }
        // even units split evenly: every part within one unit of the share
        if (trial % 10 == 0) {
            std::vector<double> e(n, 1.0);
            const std::vector<int> be = svt::split_units(e, (double)n / 7.0 * (1.0 + 1e-6), 64);
            const int pe = (int)be.size() - 1;
            expect(pe == std::min(7, n), "even split count", pe, std::min(7, n));
            for (int k = 0; k < pe; ++k)
                expect(std::fabs((be[k + 1] - be[k]) - (double)n / pe) <= 1.0 + 1e-9, "even part size",
                       be[k + 1] - be[k], n);
        }
    }
}

using Cache = std::map<svt::TuneKey, std::vector<int>>;

// Same entries (keys compared by their order: neither precedes the other).
bool same(const Cache &a, const Cache &b)
{
    if (a.size() != b.size())
        return false;
    for (auto x = a.begin(), y = b.begin(); x != a.end(); ++x, ++y)
        if (x->first < y->first || y->first < x->first || x->second != y->second)
            return false;
    return true;
}

svt::TuneKey random_key(std::mt19937_64 &rng)
{
    std::uniform_int_distribution<int> dim(1, 1 << 16), it(0, 1000), pr(0, 3), sch(0, 2), nm(0, 2),
        bit(0, 1), hp(-1, 10);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    // ell0 log-uniform in [1e-6, 0.9]
    const double ell0 = std::exp(std::log(1e-6) + u(rng) * (std::log(0.9) - std::log(1e-6)));
    return svt::TuneKey{dim(rng), dim(rng), it(rng), pr(rng), sch(rng), nm(rng), bit(rng), bit(rng), hp(rng),
                        ell0, u(rng) < 0.3 ? 0.0 : u(rng), bit(rng)};
}

void check_json(std::mt19937_64 &rng)
{
    const char *gpu = "NVIDIA GB300 \"test\" \\ name";
    const int sms = 152;
    std::uniform_int_distribution<int> cnt(0, 12), nw(1, 70), wi(0, 2);
    const int widths[3] = {128, 256, svt::kBnPair};
    for (int trial = 0; trial < 300; ++trial) {
        Cache t;
        const int c = cnt(rng);
        for (int i = 0; i < c; ++i) {
            std::vector<int> w(nw(rng));
            for (int &x : w)
                x = widths[wi(rng)];
            t[random_key(rng)] = w;
        }
        const std::string text = svt::tuning_to_json(gpu, sms, t);
        Cache back;
        expect(svt::tuning_from_json(text.c_str(), gpu, sms, &back), "reads its own output", trial);
        expect(same(back, t), "round trip", (long long)back.size(), (long long)t.size());
        // rejected: another GPU, another SM count, truncation, trailing text
        Cache keep{{random_key(rng), {128}}}, out = keep;
        expect(!svt::tuning_from_json(text.c_str(), "other", sms, &out) && same(out, keep), "other gpu");
        expect(!svt::tuning_from_json(text.c_str(), gpu, sms + 1, &out) && same(out, keep), "other sm count");
        if (text.size() > 2) {
            const std::string cut = text.substr(0, text.size() / 2);
            expect(!svt::tuning_from_json(cut.c_str(), gpu, sms, &out) && same(out, keep), "truncated");
        }
        const std::string extra = text + " x";
        expect(!svt::tuning_from_json(extra.c_str(), gpu, sms, &out) && same(out, keep), "trailing text");
    }
    // hand-written malformed and out-of-range texts
    const std::string head = std::string("{\"format\": 1, \"gpu\": \"g\", \"sms\": 2, \"entries\": [");
    auto entry = [](const std::string &widths, const std::string &ell0, const std::string &iters) {
        return "{\"m\": 4, \"n\": 4, \"iters\": " + iters + ", \"prec\": 2, \"schedule\": 1, \"norm\": 0, "
               "\"polish\": 1, \"mode\": 0, \"hp_steps\": -1, \"ell0\": " + ell0 +
               ", \"delta\": 0, \"fuse\": 1, \"widths\": [" + widths + "]}";
    };
    Cache out;
    expect(svt::tuning_from_json((head + entry("256", "0.001", "20") + "]}").c_str(), "g", 2, &out) &&
               out.size() == 1,
           "valid hand-written entry");
    const std::string bad[] = {
        head + entry("300", "0.001", "20") + "]}",        // no such tile width
        head + entry("", "0.001", "20") + "]}",           // no widths
        head + entry("256", "1.5", "20") + "]}",          // ell0 outside (0, 1)
        head + entry("256", "-nan", "20") + "]}",         // not a finite number
        head + entry("256", "0.001", "20.5") + "]}",      // not an integer
        head + entry("256", "0.001", "5000") + "]}",      // out of range
        "{\"format\": 2, \"gpu\": \"g\", \"sms\": 2, \"entries\": []}",  // another format
        "{\"gpu\": \"g\", \"sms\": 2, \"entries\": []}",                 // no format
        "{\"format\": 1, \"gpu\": \"\\u00e9\", \"sms\": 2, \"entries\": []}",  // non-ASCII escape
        "{\"format\": 1, \"gpu\": \"g\\q\", \"sms\": 2, \"entries\": []}",     // bad escape
        "[]",
        "",
        std::string(40, '[') + std::string(40, ']'),   // nested too deep
    };
    for (const std::string &b : bad) {
        Cache o{{random_key(rng), {256}}}, k = o;
        expect(!svt::tuning_from_json(b.c_str(), "g", 2, &o) && same(o, k), "rejected", (long long)b.size());
    }
}

void check_arena(std::mt19937_64 &rng)
{
    const size_t A = 256;
    std::uniform_int_distribution<int> ops(50, 400), pick(0, 1 << 30);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    for (int trial = 0; trial < 300; ++trial) {
        svt::Arena ar;
        const size_t size = A * (1 + pick(rng) % 4096);
        ar.reset(size);
        std::map<size_t, size_t> live;  // offset -> rounded length
        const int nops = ops(rng);
        for (int op = 0; op < nops; ++op) {
            if (live.empty() || u(rng) < 0.55) {
                const size_t len = 1 + (size_t)(u(rng) * u(rng) * (double)size * 0.4);
                const size_t rl = svt::Arena::round_up(len, A);
                // the model: free ranges are the gaps between live ranges
                size_t expect_off = SIZE_MAX, at = 0;
                for (const auto &kv : live) {
                    if (kv.first - at >= rl && expect_off == SIZE_MAX)
                        expect_off = at;
                    at = kv.first + kv.second;
                }
                if (expect_off == SIZE_MAX && size - at >= rl)
                    expect_off = at;
                size_t off = 0;
                const bool ok = ar.alloc(len, &off);
                expect(ok == (expect_off != SIZE_MAX), "alloc fails only when nothing fits",
                       (long long)rl, (long long)expect_off);
                if (ok) {
                    expect(off == expect_off, "first fit", (long long)off, (long long)expect_off);
                    expect(off % A == 0 && off + rl <= size, "inside the arena", (long long)off,
                           (long long)rl);
                    live[off] = rl;
                }
            } else {
                auto it = live.begin();
                std::advance(it, pick(rng) % live.size());
                ar.release(it->first, it->second);
                live.erase(it);
            }
            // live ranges disjoint; free ranges disjoint, coalesced, and the complement
            size_t prev_end = 0, free_sum = 0, live_sum = 0;
            for (const auto &kv : live) {
                expect(kv.first >= prev_end, "live ranges disjoint", (long long)kv.first,
                       (long long)prev_end);
                prev_end = kv.first + kv.second;
                live_sum += kv.second;
            }
            size_t fend = 0;
            bool first = true;
            for (const auto &kv : ar.free_) {
                expect(first || kv.first > fend, "free ranges disjoint and coalesced",
                       (long long)kv.first, (long long)fend);
                expect(live.find(kv.first) == live.end(), "free range is not live", (long long)kv.first);
                fend = kv.first + kv.second;
                free_sum += kv.second;
                first = false;
            }
            expect(free_sum + live_sum == size, "free + live = size", (long long)(free_sum + live_sum),
                   (long long)size);
        }
        for (const auto &kv : live)
            ar.release(kv.first, kv.second);
        expect(ar.free_.size() == 1 && ar.free_.begin()->first == 0 && ar.free_.begin()->second == size,
               "everything released: one range");
    }
}

} // namespace

int main(int argc, char **argv)
{
    std::mt19937_64 rng(argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 1);
    check_split(rng);
    check_json(rng);
    check_arena(rng);
    std::printf("%d failures\n", failures);
    return failures == 0 ? 0 : 1;
}
