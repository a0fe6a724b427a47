// Checks the dependencies that derive_fused_deps (fused_deps.h) gives the products of
// a fused solve, by simulation at block granularity.
//
// Every product D = L R^T is a grid of tiles; a tile reads the row strip of L at its
// tile row and the row strip of R at its tile column when it starts, and its C block
// when it ends, then writes its output block (and the mirror of a symmetric product,
// and the transposed copy). A tile may start or end only when the conditions the
// kernel checks hold (whole-problem counters, strip counters with the derived bases
// and targets, the shortcut "source complete"), and the scheduler picks among all
// tiles of all products that may move, at random: far more orders than the
// persistent kernel produces. Every read must see, block by block, exactly the
// version the program order implies (the latest earlier writer, complete), no write
// may overwrite a block that an earlier reader in program order still has to read,
// norms must be complete before a product's scales read them, and the simulation
// must never stall.
//
// Usage: fused_deps_check <seed> <rounds>; exit status 0 when every check passed.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "fused_deps.h"

using svt::DepProduct;
using svt::DepResult;

namespace {

constexpr int kPerCta = 8;  // completion increments per CTA tile

struct Buffer {
    int rows, cols;  // in blocks
};

struct Product {
    int l = -1, r = -1, c = -1, o = -1, t = -1;  // buffer ids (-1: none)
    int o_trans = 0, sym = 0, chain = 0;
    int tiles_m = 0, tiles_n = 0;
    int theta = -1, norm = -1;  // norm ids
};

struct Block {
    int buf, row, col;
    bool operator<(const Block &o) const
    {
        return buf != o.buf ? buf < o.buf : (row != o.row ? row < o.row : col < o.col);
    }
};

int failures = 0;

void fail(const char *what, int p, int extra = -1)
{
    if (failures < 20)
        std::printf("FAIL: %s (product %d, %d)\n", what, p, extra);
    ++failures;
}

// One simulated launch. Returns true when it completed.
int refused = 0;

bool simulate(const std::vector<Buffer> &bufs, const std::vector<Product> &ps, bool strips,
              int ctas, std::mt19937 &rng, bool must_fit = true)
{
    const int n = (int)ps.size();
    std::vector<DepProduct> dps(n);
    // distinct fake addresses for buffers and norms
    static char buf_addr[64], norm_addr[64];
    std::vector<std::vector<std::pair<int, int>>> tiles(n);
    for (int p = 0; p < n; ++p) {
        const Product &q = ps[p];
        for (int i = 0; i < q.tiles_m; ++i)
            for (int j = 0; j < q.tiles_n; ++j)
                if (!q.sym || i <= j)
                    tiles[p].push_back({i, j});
        auto addr = [&](int b) -> const void * { return b < 0 ? nullptr : &buf_addr[b]; };
        auto naddr = [&](int m) -> const double * {
            return m < 0 ? nullptr : reinterpret_cast<const double *>(&norm_addr[m * 8 % 64]);
        };
        dps[p] = {addr(q.l), addr(q.r), addr(q.c), addr(q.o), addr(q.t), q.o_trans, q.sym,
                  q.chain, q.tiles_m, q.tiles_n, (int)tiles[p].size() * ctas, naddr(q.theta),
                  naddr(q.norm)};
    }
    const int per_tile = kPerCta * ctas;
    std::vector<DepResult> d;
    if (!svt::derive_fused_deps(dps, strips, kPerCta, per_tile, 1 << 20, d)) {
        // more conditions than the table's slots: such a plan runs launch by launch
        if (must_fit)
            fail("derivation refused the solve's sequence", -1);
        else
            ++refused;
        return false;
    }
    // program-order expectations: the writer each read must see
    std::vector<std::map<int, int>> expect(n);  // product -> buffer -> writer (-1 ingest)
    std::map<int, int> last_writer, last_norm;
    std::vector<int> norm_src(n, -1);
    for (int p = 0; p < n; ++p) {
        const Product &q = ps[p];
        for (int b : {q.l, q.r, q.c})
            if (b >= 0)
                expect[p][b] = last_writer.count(b) ? last_writer[b] : -1;
        if (q.theta >= 0 && last_norm.count(q.theta))
            norm_src[p] = last_norm[q.theta];
        if (q.o >= 0)
            last_writer[q.o] = p;
        if (q.t >= 0)
            last_writer[q.t] = p;
        if (q.norm >= 0)
            last_norm[q.norm] = p;
    }
    // blocks each product still has to read: count of its tiles that read each block
    std::vector<std::map<Block, int>> need(n);
    auto reads_of = [&](int p, int i, int j, bool at_start) {
        const Product &q = ps[p];
        std::vector<Block> v;
        if (at_start) {
            if (q.l >= 0)
                for (int k = 0; k < bufs[q.l].cols; ++k)
                    v.push_back({q.l, i, k});
            if (q.r >= 0)
                for (int k = 0; k < bufs[q.r].cols; ++k)
                    v.push_back({q.r, j, k});
        } else if (q.c >= 0) {
            v.push_back({q.c, i, j});
        }
        return v;
    };
    auto writes_of = [&](int p, int i, int j) {
        const Product &q = ps[p];
        std::vector<Block> v;
        if (q.o >= 0) {
            v.push_back(q.o_trans ? Block{q.o, j, i} : Block{q.o, i, j});
            if (q.sym && i != j)
                v.push_back({q.o, j, i});
        }
        if (q.t >= 0)
            v.push_back({q.t, j, i});
        return v;
    };
    for (int p = 0; p < n; ++p)
        for (auto [i, j] : tiles[p])
            for (bool st : {true, false})
                for (const Block &b : reads_of(p, i, j, st))
                    ++need[p][b];
    std::map<Block, int> version;  // absent: -1 (written before the launch)
    auto ver = [&](const Block &b) {
        auto it = version.find(b);
        return it == version.end() ? -1 : it->second;
    };
    std::vector<int> state_done(n, 0);       // finished tiles per product
    std::vector<std::vector<int>> state(n);  // per tile: 0 waiting, 1 started, 2 finished
    for (int p = 0; p < n; ++p)
        state[p].assign(tiles[p].size(), 0);
    std::vector<int> strip_cnt(1 << 16, 0);
    auto whole_done = [&](int p, int target) { return state_done[p] * per_tile >= target; };
    auto strip_ok = [&](int p, int k, int idx) {
        const DepResult &r = d[p];
        if (!r.sdep_mode[k])
            return true;
        if (whole_done(r.sdep_src[k], r.sdep_whole[k]))
            return true;
        return strip_cnt[r.sdep_base[k] + idx] * per_tile >= r.sdep_target[k];
    };
    auto can_start = [&](int p, int i, int j) {
        const DepResult &r = d[p];
        for (int k = 0; k < 2; ++k)
            if (r.dep[k] >= 0 && !whole_done(r.dep[k], r.dep_target[k]))
                return false;
        return strip_ok(p, 0, i) && strip_ok(p, 1, j);
    };
    auto can_end = [&](int p, int i, int j) {
        const DepResult &r = d[p];
        const Product &q = ps[p];
        if (q.c >= 0 || q.theta >= 0)
            for (int k = 0; k < 2; ++k)
                if (r.dep[k] >= 0 && !whole_done(r.dep[k], r.dep_target[k]))
                    return false;
        for (int k = 0; k < r.nwdep; ++k)
            if (!whole_done(r.wdep[k], r.wdep_target[k]))
                return false;
        (void)j;
        return strip_ok(p, 2, i);
    };
    int remaining = 0;
    for (int p = 0; p < n; ++p)
        remaining += (int)tiles[p].size();
    std::vector<std::pair<int, int>> moves;  // (product, tile)
    while (remaining > 0) {
        moves.clear();
        for (int p = 0; p < n; ++p)
            for (int t = 0; t < (int)tiles[p].size(); ++t) {
                auto [i, j] = tiles[p][t];
                if ((state[p][t] == 0 && can_start(p, i, j)) ||
                    (state[p][t] == 1 && can_end(p, i, j)))
                    moves.push_back({p, t});
            }
        if (moves.empty()) {
            fail("simulation stalled", -1, remaining);
            return false;
        }
        auto [p, t] = moves[std::uniform_int_distribution<int>(0, (int)moves.size() - 1)(rng)];
        auto [i, j] = tiles[p][t];
        const Product &q = ps[p];
        const bool start = state[p][t] == 0;
        for (const Block &b : reads_of(p, i, j, start)) {
            if (ver(b) != expect[p][b.buf])
                fail(start ? "operand read sees the wrong version" : "C read sees the wrong version",
                     p, b.buf);
            --need[p][b];
        }
        if (start) {
            state[p][t] = 1;
            continue;
        }
        if (q.theta >= 0 && norm_src[p] >= 0 && state_done[norm_src[p]] != (int)tiles[norm_src[p]].size())
            fail("scales read an incomplete norm", p, norm_src[p]);
        for (const Block &b : writes_of(p, i, j)) {
            // the previous writer must be complete on this block ...
            int prev = -1;
            for (int w = p - 1; w >= 0; --w)
                if (ps[w].o == b.buf || ps[w].t == b.buf) {
                    prev = w;
                    break;
                }
            if (ver(b) != prev)
                fail("write overtakes the previous writer", p, b.buf);
            // ... and every earlier reader of that version done with it
            for (int r = prev + 1; r < p; ++r) {
                auto it = need[r].find(b);
                if (it != need[r].end() && it->second > 0)
                    fail("write clobbers a block an earlier reader still needs", p, r);
            }
            version[b] = p;
        }
        state[p][t] = 2;
        ++state_done[p];
        --remaining;
        const DepResult &r = d[p];
        if (r.strip_base >= 0) {
            ++strip_cnt[r.strip_base + i];
            if (!q.sym)
                ++strip_cnt[r.strip_base + q.tiles_m + j];
            else if (j != i)
                ++strip_cnt[r.strip_base + j];
        }
    }
    return true;
}

// The products of one solve, in the plan builder's order (tall problem M x N in
// blocks): Gram, per step Y, Z, X Z for the P chain and S^2, Y^2, S Z for the S chain,
// the polish of both chains and the combine. skip_p: Corollary 1's mode, no P chain (B
// is A, written before the launch).
void solve_sequence(int Tm, int T, int steps, std::vector<Buffer> &bufs, std::vector<Product> &ps,
                    bool skip_p = false)
{
    enum { X0, X1, Xt0, Xt1, S0, S1, Yp, Zp, Ys, Zs, ZPp, ZSp, B, Sp, NB };
    bufs.assign(NB, {T, T});
    bufs[X0] = bufs[X1] = bufs[B] = {Tm, T};
    bufs[Xt0] = bufs[Xt1] = {T, Tm};
    enum { NRM_S0, NRM_YP, NRM_YS, NRM_OUT };
    auto sq = [&](int l, int r, int c, int o, int chain, int theta, int norm) {
        Product q;
        q.l = l, q.r = r, q.c = c, q.o = o, q.sym = 1, q.chain = chain;
        q.tiles_m = q.tiles_n = T;
        q.theta = theta, q.norm = norm;
        ps.push_back(q);
    };
    ps.clear();
    sq(Xt0, Xt0, -1, S0, 1, -1, NRM_S0);  // Gram (its operands come from the ingest)
    int cur = 0;
    const int X[2] = {X0, X1}, Xt[2] = {Xt0, Xt1}, S[2] = {S0, S1};
    for (int s = 0; s < steps; ++s) {
        const int nxt = 1 - cur;
        if (!skip_p)
            sq(Xt[cur], Xt[cur], -1, Yp, 0, -1, s == 0 ? NRM_YP : -1);
        sq(S[cur], S[cur], -1, Ys, 1, -1, s == 0 ? NRM_YS : -1);
        if (!skip_p)
            sq(Yp, Yp, Yp, Zp, 0, s == 0 ? NRM_YP : -1, -1);
        sq(Ys, Ys, Ys, Zs, 1, s == 0 ? NRM_YS : -1, -1);
        if (!skip_p) {
            Product xz;
            xz.l = X[cur], xz.r = Zp, xz.o = X[nxt], xz.t = Xt[nxt], xz.chain = 0;
            xz.tiles_m = Tm, xz.tiles_n = T;
            ps.push_back(xz);
        }
        sq(S[cur], Zs, -1, S[nxt], 1, -1, -1);
        cur = nxt;
    }
    if (!skip_p)
        sq(Xt[cur], Xt[cur], -1, ZPp, 0, -1, -1);
    sq(S[cur], S[cur], -1, ZSp, 1, -1, -1);
    if (!skip_p) {
        Product pb;
        pb.l = X[cur], pb.r = ZPp, pb.o = B, pb.chain = 0, pb.tiles_m = Tm, pb.tiles_n = T;
        ps.push_back(pb);
    }
    sq(S[cur], ZSp, -1, Sp, 1, -1, -1);
    Product comb;  // output to the caller's Y: no buffer of the launch
    comb.l = B, comb.r = Sp, comb.c = B, comb.chain = 2, comb.tiles_m = Tm, comb.tiles_n = T;
    comb.norm = NRM_OUT;
    ps.push_back(comb);
}

// Random products over a few square buffers (strip mode must be safe for any order).
void random_sequence(std::mt19937 &rng, std::vector<Buffer> &bufs, std::vector<Product> &ps)
{
    const int T = std::uniform_int_distribution<int>(1, 4)(rng);
    const int nb = 5;
    bufs.assign(nb, {T, T});
    const int n = std::uniform_int_distribution<int>(2, 12)(rng);
    ps.clear();
    auto pick = [&](int lo, int hi) { return std::uniform_int_distribution<int>(lo, hi)(rng); };
    for (int k = 0; k < n; ++k) {
        Product q;
        q.l = pick(0, nb - 1);
        q.r = pick(0, 2) ? q.l : pick(0, nb - 1);
        q.c = pick(0, 2) ? -1 : pick(0, nb - 1);
        do {
            q.o = pick(0, nb - 1);
        } while (q.o == q.l || q.o == q.r || q.o == q.c);
        q.sym = pick(0, 1);
        q.o_trans = q.sym ? 0 : pick(0, 1);
        if (!q.sym && pick(0, 1)) {
            do {
                q.t = pick(0, nb - 1);
            } while (q.t == q.l || q.t == q.r || q.t == q.c || q.t == q.o);
        }
        q.chain = pick(0, 2);
        q.tiles_m = q.tiles_n = T;
        q.norm = pick(0, 3) ? -1 : pick(0, 1);
        q.theta = pick(0, 3) ? -1 : pick(0, 1);
        ps.push_back(q);
    }
}

} // namespace

int main(int argc, char **argv)
{
    const unsigned seed = argc > 1 ? (unsigned)std::atoi(argv[1]) : 1u;
    const int rounds = argc > 2 ? std::atoi(argv[2]) : 20;
    std::mt19937 rng(seed);
    std::vector<Buffer> bufs;
    std::vector<Product> ps;
    int sims = 0;
    // the solve's own sequence, both modes, square and tall, plain and paired tiles
    for (int shape = 0; shape < 8; ++shape) {
        const int T = 2 + shape % 2, Tm = (shape & 2) ? 2 * T : T;
        solve_sequence(Tm, T, 3, bufs, ps, shape >= 4);  // shapes 4-7: no P chain
        for (bool strips : {false, true})
            for (int ctas : {1, 2})
                for (int r = 0; r < rounds; ++r) {
                    simulate(bufs, ps, strips, ctas, rng);
                    ++sims;
                }
    }
    // arbitrary product sequences in strip mode
    for (int r = 0; r < 40 * rounds; ++r) {
        random_sequence(rng, bufs, ps);
        simulate(bufs, ps, true, 1 + (r & 1), rng, false);
        ++sims;
    }
    std::printf("%d simulations (%d random sequences over the table's slots), %d failures\n", sims,
                refused, failures);
    return failures ? 1 : 0;
}
