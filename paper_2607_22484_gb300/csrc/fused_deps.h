// Dependencies between the products of one fused solve (host code only: no CUDA
// calls, so that it can be checked on its own).
//
// A fused solve runs every product of the method (Section 2: the shifted Gram, the
// polynomial steps of both polar chains, the polish and the combine of
// Proposition 1) in one persistent launch; tiles of later products start while
// earlier ones are still running, so each product carries the conditions under
// which its tiles may read and write:
//
// * chain mode (strips = false): every product waits for the whole previous
//   product of its chain (P or S; the combine for both). The chains only read what
//   their own earlier products or the ingest wrote, so this orders every access.
// * strip mode (strips = true, square tiles): from the buffers each product reads
//   and writes. A read of a buffer written earlier in the launch waits for the
//   strip it reads: rows of L for the tile's row, rows of R for its column, the C
//   block's row; a strip of a row-major output is one tile row, of a transposed
//   output one tile column, of a symmetric product the rows and columns of one
//   index. Before its stores a tile waits for every earlier reader (WAR) and writer
//   (WAW) of the buffers it overwrites, and for the product that accumulates a norm
//   its scales are computed from.
#pragma once

#include <map>
#include <vector>

namespace svt {

// One product D = L R^T as the derivation sees it.
struct DepProduct {
    const void *l, *r, *c;  // buffers read (hi parts; null: none, or the caller's)
    const void *o, *t;      // buffers written: the output, the transposed copy
    int o_trans;            // the output is stored transposed
    int sym;                // symmetric product: upper tiles, mirrored output
    int chain;              // 0 P chain, 1 S chain, 2 both (the combine)
    int tiles_m, tiles_n;   // tile grid
    int valid;              // CTA tiles with work (the completion-count unit)
    const double *theta_src, *norm_acc;  // norm read by the scales / accumulated
    const void *f = nullptr;  // written: an extra copy in the output's orientation (e4m3)
};

// What one product waits for (the fields of the same names in TcProblem).
struct DepResult {
    int dep[2] = {-1, -1}, dep_target[2] = {0, 0};
    int nwdep = 0, wdep[4] = {0, 0, 0, 0}, wdep_target[4] = {0, 0, 0, 0};
    int sdep_mode[3] = {0, 0, 0}, sdep_base[3] = {0, 0, 0}, sdep_target[3] = {0, 0, 0};
    int sdep_src[3] = {0, 0, 0}, sdep_whole[3] = {0, 0, 0};
    int strip_base = -1;
};

// per_cta: completion increments per CTA tile (epilogue warps); per_tile: per
// scheduled tile (per_cta x CTAs per tile); strip_capacity: strip counters
// available. Returns false when the conditions do not fit the table's slots.
inline bool derive_fused_deps(const std::vector<DepProduct> &ps, bool strips, int per_cta,
                              int per_tile, int strip_capacity, std::vector<DepResult> &out)
{
    out.assign(ps.size(), DepResult());
    struct Writer {
        int pid, mode;  // mode: 1 row-major output, 2 transposed output, 3 symmetric
    };
    std::map<const void *, Writer> writers;
    std::map<const void *, std::vector<int>> readers;
    std::map<const double *, int> norm_writer;
    int lastp[2] = {-1, -1};
    int strip_next = 0;
    for (int pid = 0; pid < (int)ps.size(); ++pid) {
        const DepProduct &p = ps[pid];
        DepResult &d = out[pid];
        if (!strips) {
            if (p.chain < 2) {
                d.dep[0] = lastp[p.chain];
            } else {
                d.dep[0] = lastp[0];
                d.dep[1] = lastp[1];
            }
            for (int k = 0; k < 2; ++k)
                if (d.dep[k] >= 0)
                    d.dep_target[k] = per_cta * ps[d.dep[k]].valid;
            if (p.chain < 2)
                lastp[p.chain] = pid;
            else
                lastp[0] = lastp[1] = pid;
            continue;
        }
        d.strip_base = strip_next;
        strip_next += p.sym ? p.tiles_n : p.tiles_m + p.tiles_n;
        if (strip_next > strip_capacity)
            return false;
        bool ok = true;
        auto before_store = [&](int w) {
            if (w < 0 || w == pid)
                return;
            for (int k = 0; k < d.nwdep; ++k)
                if (d.wdep[k] == w)
                    return;
            if (d.nwdep < 4)
                d.wdep[d.nwdep++] = w;
            else
                ok = false;
        };
        // RAW: L and R (read before the MMAs), C (read by the epilogue)
        const void *in[3] = {p.l, p.r, p.c};
        for (int k = 0; k < 3; ++k) {
            if (!in[k])
                continue;
            auto it = writers.find(in[k]);
            if (it == writers.end())
                continue;  // written before this launch
            const Writer w = it->second;
            const DepProduct &src = ps[w.pid];
            d.sdep_mode[k] = w.mode;
            d.sdep_base[k] = out[w.pid].strip_base + (w.mode == 2 ? src.tiles_m : 0);
            d.sdep_target[k] = per_tile * (w.mode == 2 ? src.tiles_m : src.tiles_n);
            d.sdep_src[k] = w.pid;
            d.sdep_whole[k] = per_cta * src.valid;
        }
        // the norm the scales are computed from
        if (p.theta_src) {
            auto it = norm_writer.find(p.theta_src);
            if (it != norm_writer.end())
                before_store(it->second);
        }
        // WAR / WAW on the buffers this product writes
        const void *outs[3] = {p.o, p.t, p.f};
        for (const void *b : outs) {
            if (!b)
                continue;
            auto rd = readers.find(b);
            if (rd != readers.end())
                for (int r : rd->second)
                    before_store(r);
            auto wr = writers.find(b);
            if (wr != writers.end())
                before_store(wr->second.pid);
        }
        if (!ok)
            return false;
        for (int k = 0; k < d.nwdep; ++k)
            d.wdep_target[k] = per_cta * ps[d.wdep[k]].valid;
        // record this product's reads and writes
        for (int k = 0; k < 3; ++k)
            if (in[k])
                readers[in[k]].push_back(pid);
        if (p.o) {
            writers[p.o] = {pid, p.sym ? 3 : (p.o_trans ? 2 : 1)};
            readers[p.o].clear();
        }
        if (p.t) {
            writers[p.t] = {pid, 2};
            readers[p.t].clear();
        }
        if (p.f) {
            writers[p.f] = {pid, p.sym ? 3 : 1};
            readers[p.f].clear();
        }
        if (p.norm_acc)
            norm_writer[p.norm_acc] = pid;
    }
    return true;
}

} // namespace svt
