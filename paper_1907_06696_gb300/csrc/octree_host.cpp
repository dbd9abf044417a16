// octree_host.cpp -- host construction of adaptive octree meshes and of every table the
// device path needs (active DoFs with hanging-node constraints, local-smoothing levels,
// viscosity, right-hand side), for the adaptive sinker configuration (Abstract; Section 2.3;
// local smoothing by citation of Janssen & Kanschat, Section 2.2.1).
//
// Readings: a leaf is split while its level is below a sinker's maximum level and its
// distance interval [min, max |x - c|] over the cell box meets (r - w, r + w); the tree is then
// 2:1 balanced across faces, edges and vertices. A node of a leaf lying on a face or edge of a
// coarser neighbouring leaf, and not one of that leaf's nodes, is hanging: its value is the
// coarser leaf's Q2 (velocity) or Q1 (pressure) interpolant there; nodes on the cube boundary
// are Dirichlet instead. Level l of the hierarchy holds every cell of level l; its nodes on the
// boundary of those cells' union but inside the cube are refinement-edge nodes.
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "octree.cuh"

namespace stk {

namespace {

const int kDirs[26][3] = {{-1, -1, -1}, {0, -1, -1}, {1, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {1, 0, -1}, {-1, 1, -1},
                          {0, 1, -1},   {1, 1, -1},  {-1, -1, 0}, {0, -1, 0},  {1, -1, 0}, {-1, 0, 0},  {1, 0, 0},
                          {-1, 1, 0},   {0, 1, 0},   {1, 1, 0},   {-1, -1, 1}, {0, -1, 1}, {1, -1, 1},  {-1, 0, 1},
                          {0, 0, 1},    {1, 0, 1},   {-1, 1, 1},  {0, 1, 1},   {1, 1, 1}};

uint64_t parent_key(uint64_t c) { return oct_key(oct_l(c) - 1, oct_i(c) >> 1, oct_j(c) >> 1, oct_k(c) >> 1); }

void children_of(uint64_t c, uint64_t out[8]) {
    const int l = oct_l(c), i = oct_i(c), j = oct_j(c), k = oct_k(c);
    for (int q = 0; q < 8; ++q) out[q] = oct_key(l + 1, 2 * i + (q & 1), 2 * j + ((q >> 1) & 1), 2 * k + (q >> 2));
}

unsigned host_threads() {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    return nt > 32 ? 32 : nt;
}

template <typename F>
void parallel_for(size_t n, F f) {
    unsigned nt = host_threads();
    if (n < 4096) nt = 1;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (size_t i = n * t / nt; i < n * (t + 1) / nt; ++i) f(i);
        });
    for (auto& x : th) x.join();
}

// Sort with the host threads: chunks sorted in parallel, then merged pairwise. For a total order
// (elements that compare equal are identical) the result equals std::sort's.
template <typename T, typename Less = std::less<T>>
void par_sort(std::vector<T>& v, Less less = Less()) {
    size_t P = 1;
    while (2 * P <= host_threads()) P *= 2;
    if (P == 1 || v.size() < (size_t(1) << 16)) {
        std::sort(v.begin(), v.end(), less);
        return;
    }
    std::vector<size_t> b(P + 1);
    for (size_t i = 0; i <= P; ++i) b[i] = v.size() * i / P;
    {
        std::vector<std::thread> th;
        for (size_t i = 0; i < P; ++i) th.emplace_back([&, i] { std::sort(v.begin() + b[i], v.begin() + b[i + 1], less); });
        for (auto& x : th) x.join();
    }
    std::vector<T> tmp(v.size());
    for (size_t w = 1; w < P; w *= 2) {
        std::vector<std::thread> th;
        for (size_t i = 0; i < P; i += 2 * w)
            th.emplace_back([&, i] {
                const size_t lo = b[i], mid = b[std::min(i + w, P)], hi = b[std::min(i + 2 * w, P)];
                std::merge(v.begin() + lo, v.begin() + mid, v.begin() + mid, v.begin() + hi, tmp.begin() + lo, less);
            });
        for (auto& x : th) x.join();
        v.swap(tmp);
    }
}

// Runs f(i) for i < n on the host threads; f returns an error message or nullptr. Returns the
// message of the smallest failing i (the one a sequential loop would report), or nullptr.
template <typename F>
const char* parallel_check(size_t n, F f) {
    std::vector<const char*> err(n, nullptr);
    parallel_for(n, [&](size_t i) { err[i] = f(i); });
    for (size_t i = 0; i < n; ++i)
        if (err[i]) return err[i];
    return nullptr;
}

// Quadratic Lagrange basis on {0, 1/2, 1} at the lattice positions 0, 1/4, 1/2, 3/4, 1.
const double kQ2At[5][3] = {{1, 0, 0}, {0.375, 0.75, -0.125}, {0, 1, 0}, {-0.125, 0.75, 0.375}, {0, 0, 1}};

double lag(int m, double x) {
    return m == 0 ? 2.0 * (x - 0.5) * (x - 1.0) : m == 1 ? -4.0 * x * (x - 1.0) : 2.0 * x * (x - 0.5);
}

}  // namespace

std::vector<uint64_t> oct_refine_shells(int base_level, int n_sinkers, const double* centres, const int* max_levels,
                                        double radius, double half_width) {
    const int n = 1 << base_level;
    std::vector<uint64_t> leaves;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) leaves.push_back(oct_key(base_level, i, j, k));
    const double lo_r = radius - half_width, hi_r = radius + half_width;
    bool changed = true;
    while (changed) {
        changed = false;
        std::vector<uint64_t> nxt;
        nxt.reserve(leaves.size() * 2);
        for (uint64_t c : leaves) {
            const int l = oct_l(c);
            const double h = std::ldexp(1.0, -l);
            const double lo[3] = {oct_i(c) * h, oct_j(c) * h, oct_k(c) * h};
            bool split = false;
            for (int s = 0; s < n_sinkers && !split; ++s) {
                if (l >= max_levels[s]) continue;
                double dmin2 = 0.0, dmax2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double a = lo[d], b = lo[d] + h, x = centres[3 * s + d];
                    const double gap = std::max(std::max(a - x, 0.0), x - b);
                    const double far = std::max(std::fabs(x - a), std::fabs(x - b));
                    dmin2 = dmin2 + gap * gap;
                    dmax2 = dmax2 + far * far;
                }
                if (std::sqrt(dmin2) < hi_r && std::sqrt(dmax2) > lo_r) split = true;
            }
            if (split) {
                uint64_t ch[8];
                children_of(c, ch);
                nxt.insert(nxt.end(), ch, ch + 8);
                changed = true;
            } else {
                nxt.push_back(c);
            }
        }
        leaves.swap(nxt);
    }
    par_sort(leaves);
    return leaves;
}

std::vector<uint64_t> oct_balance(const std::vector<uint64_t>& in) {
    std::unordered_set<uint64_t> leaves(in.begin(), in.end()), cells;
    int lmax = 0;
    for (uint64_t c : in) {
        lmax = std::max(lmax, oct_l(c));
        uint64_t a = c;
        while (cells.insert(a).second && oct_l(a) > 0) a = parent_key(a);
    }
    // Finest level first: every level-(l-1) cell that touches a level-l leaf must exist; a missing
    // one is created by splitting its nearest existing ancestor (recursively). Splits only create
    // cells of level < l, so the scan of level l reads the sets while they are unchanged (in
    // parallel) and the splits follow in the scan's order. The result is the unique coarsest
    // balanced refinement of the input.
    for (int l = lmax; l >= 2; --l) {
        std::vector<uint64_t> cur;
        for (uint64_t c : leaves)
            if (oct_l(c) == l) cur.push_back(c);
        par_sort(cur);
        const int n = 1 << l;
        std::vector<std::vector<uint64_t>> miss(cur.size());
        parallel_for(cur.size(), [&](size_t t) {
            const uint64_t c = cur[t];
            for (const auto& d : kDirs) {
                const int ni = oct_i(c) + d[0], nj = oct_j(c) + d[1], nk = oct_k(c) + d[2];
                if (ni < 0 || nj < 0 || nk < 0 || ni >= n || nj >= n || nk >= n) continue;
                const uint64_t target = oct_key(l - 1, ni >> 1, nj >> 1, nk >> 1);
                if (!cells.count(target)) miss[t].push_back(target);
            }
        });
        for (const auto& list : miss)
            for (uint64_t target : list)
                while (!cells.count(target)) {
                    uint64_t anc = parent_key(target);
                    while (!cells.count(anc)) anc = parent_key(anc);
                    leaves.erase(anc);
                    uint64_t ch[8];
                    children_of(anc, ch);
                    for (uint64_t x : ch) {
                        leaves.insert(x);
                        cells.insert(x);
                    }
                }
    }
    std::vector<uint64_t> out(leaves.begin(), leaves.end());
    par_sort(out);
    return out;
}

std::string oct_build(const std::vector<uint64_t>& leaves_in, int coarsest, const OctSinkers& sk, OctHost& o,
                      bool active_only) {
    o = OctHost();
    if (leaves_in.empty()) return "no leaves";
    o.leaves = leaves_in;
    par_sort(o.leaves);
    if (std::adjacent_find(o.leaves.begin(), o.leaves.end()) != o.leaves.end()) return "duplicate leaves";
    std::unordered_set<uint64_t> leafset(o.leaves.begin(), o.leaves.end()), cells;
    int lmax = 0, lmin = 99;
    double vol = 0.0;
    for (uint64_t c : o.leaves) {
        const int l = oct_l(c);
        if (l > 15 || oct_i(c) >= (1 << l) || oct_j(c) >= (1 << l) || oct_k(c) >= (1 << l)) return "bad leaf key";
        lmax = std::max(lmax, l);
        lmin = std::min(lmin, l);
        vol += std::ldexp(1.0, -3 * l);
        uint64_t a = c;
        while (oct_l(a) > 0) {
            a = parent_key(a);
            if (leafset.count(a)) return "a leaf contains another leaf";
            if (!cells.insert(a).second) break;
        }
    }
    for (uint64_t c : o.leaves) cells.insert(c);
    if (std::fabs(vol - 1.0) > 1e-12) return "leaves do not tile the unit cube";
    if (coarsest < 0 || coarsest > lmin) return "coarsest level above the coarsest leaf";
    o.lmax = lmax;
    o.coarsest = coarsest;
    o.base = lmin;
    const uint64_t Mx = (uint64_t(1) << (lmax + 1)) + 1;
    o.Mx = Mx;
    auto S = [&](int l) { return int64_t(1) << (lmax + 1 - l); };
    auto pkey = [&](int64_t x, int64_t y, int64_t z) { return uint64_t(x) + Mx * (uint64_t(y) + Mx * uint64_t(z)); };
    auto on_bnd = [&](int64_t x, int64_t y, int64_t z) {
        const int64_t t = int64_t(Mx) - 1;
        return x == 0 || y == 0 || z == 0 || x == t || y == t || z == t;
    };
    const size_t nl = o.leaves.size();

    // ---- coarser neighbours of every leaf: (leaf, direction, coarse leaf)
    struct CN {
        uint32_t leaf;
        int8_t d[3];
        uint64_t coarse;
    };
    std::vector<CN> cn;
    for (size_t n = 0; n < nl; ++n) {
        const uint64_t c = o.leaves[n];
        const int l = oct_l(c), N = 1 << l;
        for (const auto& d : kDirs) {
            const int ni = oct_i(c) + d[0], nj = oct_j(c) + d[1], nk = oct_k(c) + d[2];
            if (ni < 0 || nj < 0 || nk < 0 || ni >= N || nj >= N || nk >= N) continue;
            if (cells.count(oct_key(l, ni, nj, nk))) continue;
            const uint64_t coarse = oct_key(l - 1, ni >> 1, nj >> 1, nk >> 1);
            if (!leafset.count(coarse)) return "mesh is not 2:1 balanced";
            cn.push_back({uint32_t(n), {int8_t(d[0]), int8_t(d[1]), int8_t(d[2])}, coarse});
        }
    }
    auto on_side = [](const int loc[3], const int8_t d[3], int top) {
        for (int q = 0; q < 3; ++q) {
            if (d[q] == 1 && loc[q] != top) return false;
            if (d[q] == -1 && loc[q] != 0) return false;
        }
        return true;
    };

    // ---- velocity nodes
    {
        std::vector<std::pair<uint64_t, int>> all(nl * 27);
        parallel_for(nl, [&](size_t n) {
            const uint64_t c = o.leaves[n];
            const int l = oct_l(c);
            const int64_t s = S(l), h2 = s / 2;
            for (int a = 0; a < 27; ++a)
                all[n * 27 + a] = {pkey(oct_i(c) * s + (a % 3) * h2, oct_j(c) * s + ((a / 3) % 3) * h2,
                                        oct_k(c) * s + (a / 9) * h2), l};
        });
        par_sort(all);
        std::vector<std::pair<uint64_t, int>> nodes;   // key, coarsest leaf level
        for (auto& p : all)
            if (nodes.empty() || nodes.back().first != p.first) nodes.push_back(p);
        std::vector<std::pair<uint64_t, uint64_t>> hang;   // key, coarse leaf
        for (const CN& e : cn) {
            const uint64_t c = o.leaves[e.leaf];
            const int64_t s = S(oct_l(c)), h2 = s / 2;
            for (int a = 0; a < 27; ++a) {
                const int loc[3] = {a % 3, (a / 3) % 3, a / 9};
                if (!on_side(loc, e.d, 2)) continue;
                const int64_t x = oct_i(c) * s + loc[0] * h2, y = oct_j(c) * s + loc[1] * h2,
                              z = oct_k(c) * s + loc[2] * h2;
                if (on_bnd(x, y, z)) continue;
                if (x % s == 0 && y % s == 0 && z % s == 0) continue;
                hang.push_back({pkey(x, y, z), e.coarse});
            }
        }
        par_sort(hang);
        hang.erase(std::unique(hang.begin(), hang.end(),
                               [](const auto& a, const auto& b) { return a.first == b.first; }),
                   hang.end());
        size_t hp = 0;
        for (auto& p : nodes) {
            while (hp < hang.size() && hang[hp].first < p.first) ++hp;
            if (hp < hang.size() && hang[hp].first == p.first) continue;
            o.unodes.push_back(p.first);
            o.copy_level.push_back(p.second);
        }
        const size_t nu = o.unodes.size();
        o.ubnd.resize(nu);
        parallel_for(nu, [&](size_t n) {
            const uint64_t kx = o.unodes[n] % Mx, ky = (o.unodes[n] / Mx) % Mx, kz = o.unodes[n] / (Mx * Mx);
            o.ubnd[n] = on_bnd(int64_t(kx), int64_t(ky), int64_t(kz)) ? 1 : 0;
        });
        auto uidx = [&](uint64_t key) -> int64_t {
            auto it = std::lower_bound(o.unodes.begin(), o.unodes.end(), key);
            return (it != o.unodes.end() && *it == key) ? int64_t(it - o.unodes.begin()) : -1;
        };
        o.ucon_node.assign(hang.size() * kOctUCon, -1);
        o.ucon_w.assign(hang.size() * kOctUCon, 0.0);
        const char* err = parallel_check(hang.size(), [&](size_t h) -> const char* {
            const uint64_t key = hang[h].first, C = hang[h].second;
            const int64_t px = int64_t(key % Mx), py = int64_t((key / Mx) % Mx), pz = int64_t(key / (Mx * Mx));
            const int64_t s = S(oct_l(C)), q4 = s / 4;   // coarse cell side s, nodes every s/2
            const int qx = int((px - oct_i(C) * s) / q4), qy = int((py - oct_j(C) * s) / q4),
                      qz = int((pz - oct_k(C) * s) / q4);
            int t = 0;
            for (int b = 0; b < 27; ++b) {
                const double w = kQ2At[qx][b % 3] * kQ2At[qy][(b / 3) % 3] * kQ2At[qz][b / 9];
                if (w == 0.0) continue;
                const int64_t node = uidx(pkey(oct_i(C) * s + (b % 3) * (s / 2), oct_j(C) * s + ((b / 3) % 3) * (s / 2),
                                               oct_k(C) * s + (b / 9) * (s / 2)));
                if (node < 0) return "velocity constraint chain";
                if (t >= kOctUCon) return "velocity constraint with too many terms";
                o.ucon_node[h * kOctUCon + t] = int32_t(node);
                o.ucon_w[h * kOctUCon + t] = w;
                ++t;
            }
            return nullptr;
        });
        if (err) return err;
        o.leaf_u.resize(nl * 27);
        err = parallel_check(nl, [&](size_t n) -> const char* {
            const uint64_t c = o.leaves[n];
            const int64_t s = S(oct_l(c)), h2 = s / 2;
            for (int a = 0; a < 27; ++a) {
                const uint64_t key = pkey(oct_i(c) * s + (a % 3) * h2, oct_j(c) * s + ((a / 3) % 3) * h2,
                                          oct_k(c) * s + (a / 9) * h2);
                const int64_t idx = uidx(key);
                if (idx >= 0) {
                    o.leaf_u[n * 27 + a] = int32_t(idx);
                } else {
                    auto it = std::lower_bound(hang.begin(), hang.end(), std::make_pair(key, uint64_t(0)));
                    if (it == hang.end() || it->first != key) return "node neither active nor hanging";
                    o.leaf_u[n * 27 + a] = -int32_t(it - hang.begin()) - 1;
                }
            }
            return nullptr;
        });
        if (err) return err;
    }
    if (active_only) {   // the velocity space and leaf sizes are all the gradient indicator needs
        o.leaf_h.resize(nl);
        for (size_t n = 0; n < nl; ++n) o.leaf_h[n] = std::ldexp(1.0, -oct_l(o.leaves[n]));
        return "";
    }

    // ---- pressure vertices
    {
        std::vector<uint64_t> all(nl * 8);
        parallel_for(nl, [&](size_t n) {
            const uint64_t c = o.leaves[n];
            const int64_t s = S(oct_l(c));
            for (int a = 0; a < 8; ++a)
                all[n * 8 + a] = pkey((oct_i(c) + (a & 1)) * s, (oct_j(c) + ((a >> 1) & 1)) * s, (oct_k(c) + (a >> 2)) * s);
        });
        par_sort(all);
        all.erase(std::unique(all.begin(), all.end()), all.end());
        std::vector<std::pair<uint64_t, uint64_t>> hang;
        for (const CN& e : cn) {
            const uint64_t c = o.leaves[e.leaf];
            const int64_t s = S(oct_l(c));
            for (int a = 0; a < 8; ++a) {
                const int loc[3] = {a & 1, (a >> 1) & 1, a >> 2};
                if (!on_side(loc, e.d, 1)) continue;
                const int64_t x = (oct_i(c) + loc[0]) * s, y = (oct_j(c) + loc[1]) * s, z = (oct_k(c) + loc[2]) * s;
                if (x % (2 * s) == 0 && y % (2 * s) == 0 && z % (2 * s) == 0) continue;
                hang.push_back({pkey(x, y, z), e.coarse});
            }
        }
        par_sort(hang);
        hang.erase(std::unique(hang.begin(), hang.end(),
                               [](const auto& a, const auto& b) { return a.first == b.first; }),
                   hang.end());
        size_t hp = 0;
        for (uint64_t k : all) {
            while (hp < hang.size() && hang[hp].first < k) ++hp;
            if (hp < hang.size() && hang[hp].first == k) continue;
            o.pverts.push_back(k);
        }
        auto pidx = [&](uint64_t key) -> int64_t {
            auto it = std::lower_bound(o.pverts.begin(), o.pverts.end(), key);
            return (it != o.pverts.end() && *it == key) ? int64_t(it - o.pverts.begin()) : -1;
        };
        o.pcon_node.assign(hang.size() * kOctPCon, -1);
        o.pcon_w.assign(hang.size() * kOctPCon, 0.0);
        const char* err = parallel_check(hang.size(), [&](size_t h) -> const char* {
            const uint64_t key = hang[h].first, C = hang[h].second;
            const int64_t px = int64_t(key % Mx), py = int64_t((key / Mx) % Mx), pz = int64_t(key / (Mx * Mx));
            const int64_t s = S(oct_l(C)), half = s / 2;
            const int q[3] = {int((px - oct_i(C) * s) / half), int((py - oct_j(C) * s) / half),
                              int((pz - oct_k(C) * s) / half)};   // 0, 1, 2 = 0, 1/2, 1
            int t = 0;
            for (int b = 0; b < 8; ++b) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) {
                    const double xi = 0.5 * q[d];
                    w = w * (((b >> d) & 1) ? xi : 1.0 - xi);
                }
                if (w == 0.0) continue;
                const int64_t v = pidx(pkey((oct_i(C) + (b & 1)) * s, (oct_j(C) + ((b >> 1) & 1)) * s,
                                            (oct_k(C) + (b >> 2)) * s));
                if (v < 0) return "pressure constraint chain";
                if (t >= kOctPCon) return "pressure constraint with too many terms";
                o.pcon_node[h * kOctPCon + t] = int32_t(v);
                o.pcon_w[h * kOctPCon + t] = w;
                ++t;
            }
            return nullptr;
        });
        if (err) return err;
        o.leaf_p.resize(nl * 8);
        err = parallel_check(nl, [&](size_t n) -> const char* {
            const uint64_t c = o.leaves[n];
            const int64_t s = S(oct_l(c));
            for (int a = 0; a < 8; ++a) {
                const uint64_t key = pkey((oct_i(c) + (a & 1)) * s, (oct_j(c) + ((a >> 1) & 1)) * s, (oct_k(c) + (a >> 2)) * s);
                const int64_t idx = pidx(key);
                if (idx >= 0) {
                    o.leaf_p[n * 8 + a] = int32_t(idx);
                } else {
                    auto it = std::lower_bound(hang.begin(), hang.end(), std::make_pair(key, uint64_t(0)));
                    if (it == hang.end() || it->first != key) return "vertex neither active nor hanging";
                    o.leaf_p[n * 8 + a] = -int32_t(it - hang.begin()) - 1;
                }
            }
            return nullptr;
        });
        if (err) return err;
    }

    // ---- leaf viscosity (harmonic average over the Gauss points, Section 2.3) and F (Section 3.2)
    const double g[3] = {0.5 - std::sqrt(15.0) / 10.0, 0.5, 0.5 + std::sqrt(15.0) / 10.0};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    o.leaf_mu.resize(nl);
    o.leaf_h.resize(nl);
    std::vector<double> Fe(nl * 27, 0.0);   // z-component element vectors
    parallel_for(nl, [&](size_t n) {
        const uint64_t c = o.leaves[n];
        const double h = std::ldexp(1.0, -oct_l(c));
        o.leaf_h[n] = h;
        double wsum = 0.0, winv = 0.0;
        double fz[27], wq[27];
        for (int q = 0; q < 27; ++q) {
            const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
            const double x[3] = {oct_i(c) * h + h * g[qx], oct_j(c) * h + h * g[qy], oct_k(c) * h + h * g[qz]};
            double chi = 1.0;
            for (int s = 0; s < sk.n; ++s) {
                double d2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double t = x[d] - sk.centres[3 * s + d];
                    d2 = d2 + t * t;
                }
                const double m = std::max(0.0, std::sqrt(d2) - sk.omega / 2.0);
                chi = chi * (1.0 - std::exp(-sk.delta * m * m));
            }
            const double mu = chi * sk.mu_min + (1.0 - chi) * sk.mu_max;
            const double w = gw[qx] * gw[qy] * gw[qz];
            wq[q] = w;
            wsum += w;
            winv += w / mu;
            fz[q] = sk.beta * (chi - 1.0);
        }
        o.leaf_mu[n] = wsum / winv;
        for (int a = 0; a < 27; ++a) {
            double v = 0.0;
            for (int q = 0; q < 27; ++q)
                v += h * h * h * wq[q] * fz[q] * lag(a % 3, g[q % 3]) * lag((a / 3) % 3, g[(q / 3) % 3]) *
                     lag(a / 9, g[q / 9]);
            Fe[n * 27 + a] = v;
        }
    });
    const size_t nu = o.unodes.size();
    o.F.assign(3 * nu, 0.0);
    for (size_t n = 0; n < nl; ++n)
        for (int a = 0; a < 27; ++a) {
            const int32_t r = o.leaf_u[n * 27 + a];
            if (r >= 0) {
                o.F[2 * nu + r] += Fe[n * 27 + a];
            } else {
                const size_t h = size_t(-r - 1);
                for (int t = 0; t < kOctUCon; ++t)
                    if (o.ucon_node[h * kOctUCon + t] >= 0)
                        o.F[2 * nu + o.ucon_node[h * kOctUCon + t]] += o.ucon_w[h * kOctUCon + t] * Fe[n * 27 + a];
            }
        }
    for (size_t n = 0; n < nu; ++n)
        if (o.ubnd[n])
            for (int c = 0; c < 3; ++c) o.F[c * nu + n] = 0.0;

    // ---- pressure mass diagonal (with constraints) and weights int psi_a
    {
        const size_t np = o.pverts.size();
        o.mp_diag.assign(np, 0.0);
        o.p_weights.assign(np, 0.0);
        // The terms each leaf adds (to int psi_a and to the diagonal of M_p) are found in parallel
        // and then added in leaf order, so the sums equal those of a sequential loop bit for bit.
        struct Term {
            int32_t idx;
            double v;
        };
        auto leaf_terms = [&](size_t n, Term* pw, Term* md, uint32_t& npw, uint32_t& nmd) {
            npw = nmd = 0;
            const double h = o.leaf_h[n], sc = h * h * h / o.leaf_mu[n];
            int32_t idx[8][kOctPCon];
            double w[8][kOctPCon];
            for (int a = 0; a < 8; ++a) {
                const int32_t r = o.leaf_p[n * 8 + a];
                for (int t = 0; t < kOctPCon; ++t) {
                    idx[a][t] = -1;
                    w[a][t] = 0.0;
                }
                if (r >= 0) {
                    idx[a][0] = r;
                    w[a][0] = 1.0;
                } else {
                    const size_t hh = size_t(-r - 1);
                    for (int t = 0; t < kOctPCon; ++t) {
                        idx[a][t] = o.pcon_node[hh * kOctPCon + t];
                        w[a][t] = o.pcon_w[hh * kOctPCon + t];
                    }
                }
                for (int t = 0; t < kOctPCon; ++t)
                    if (idx[a][t] >= 0) {
                        if (pw) pw[npw] = {idx[a][t], w[a][t] * h * h * h / 8.0};
                        ++npw;
                    }
            }
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b) {
                    double m = 1.0;
                    for (int d = 0; d < 3; ++d) m *= (((a >> d) & 1) == ((b >> d) & 1)) ? 1.0 / 3.0 : 1.0 / 6.0;
                    for (int t = 0; t < kOctPCon; ++t)
                        for (int u = 0; u < kOctPCon; ++u)
                            if (idx[a][t] >= 0 && idx[a][t] == idx[b][u]) {
                                if (md) md[nmd] = {idx[a][t], sc * m * w[a][t] * w[b][u]};
                                ++nmd;
                            }
                }
        };
        std::vector<uint32_t> cpw(nl), cmd(nl);
        parallel_for(nl, [&](size_t n) { leaf_terms(n, nullptr, nullptr, cpw[n], cmd[n]); });
        std::vector<size_t> opw(nl + 1, 0), omd(nl + 1, 0);
        for (size_t n = 0; n < nl; ++n) {
            opw[n + 1] = opw[n] + cpw[n];
            omd[n + 1] = omd[n] + cmd[n];
        }
        std::vector<Term> tpw(opw[nl]), tmd(omd[nl]);
        parallel_for(nl, [&](size_t n) {
            uint32_t a, b;
            leaf_terms(n, tpw.data() + opw[n], tmd.data() + omd[n], a, b);
        });
        for (const Term& t : tpw) o.p_weights[size_t(t.idx)] += t.v;
        for (const Term& t : tmd) o.mp_diag[size_t(t.idx)] += t.v;
    }

    // ---- levels coarsest .. lmax
    std::unordered_map<uint64_t, double> mu_cell;
    for (size_t n = 0; n < nl; ++n) mu_cell[o.leaves[n]] = o.leaf_mu[n];
    std::vector<std::vector<uint64_t>> by_level(lmax + 1);
    for (uint64_t c : cells) by_level[oct_l(c)].push_back(c);
    for (auto& v : by_level) par_sort(v);
    for (int l = lmax; l >= 0; --l)
        for (uint64_t c : by_level[l])
            if (!mu_cell.count(c)) {
                uint64_t ch[8];
                children_of(c, ch);
                double s = 0.0;
                for (uint64_t x : ch) s += mu_cell.at(x);
                mu_cell[c] = s / 8.0;
            }
    o.levels.resize(lmax - coarsest + 1);
    for (int l = coarsest; l <= lmax; ++l) {
        OctLevelHost& L = o.levels[l - coarsest];
        L.l = l;
        L.cells = by_level[l];
        const int64_t s = S(l), h2 = s / 2;
        std::vector<uint64_t> keys(L.cells.size() * 27);
        parallel_for(L.cells.size(), [&](size_t n) {
            const uint64_t c = L.cells[n];
            for (int a = 0; a < 27; ++a)
                keys[n * 27 + a] = pkey(oct_i(c) * s + (a % 3) * h2, oct_j(c) * s + ((a / 3) % 3) * h2,
                                        oct_k(c) * s + (a / 9) * h2);
        });
        L.cell_nodes.resize(keys.size());
        std::vector<uint64_t> sorted = keys;
        par_sort(sorted);
        sorted.erase(std::unique(sorted.begin(), sorted.end()), sorted.end());
        L.nodes = sorted;
        parallel_for(keys.size(), [&](size_t t) {
            L.cell_nodes[t] = int32_t(std::lower_bound(L.nodes.begin(), L.nodes.end(), keys[t]) - L.nodes.begin());
        });
        L.mu.resize(L.cells.size());
        parallel_for(L.cells.size(), [&](size_t n) { L.mu[n] = mu_cell.at(L.cells[n]); });
        const int N = 1 << l;
        L.flags.assign(L.nodes.size(), 0);
        parallel_for(L.nodes.size(), [&](size_t t) {
            const int64_t p[3] = {int64_t(L.nodes[t] % Mx), int64_t((L.nodes[t] / Mx) % Mx), int64_t(L.nodes[t] / (Mx * Mx))};
            if (on_bnd(p[0], p[1], p[2])) {
                L.flags[t] = 1;
                return;
            }
            int lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                const int64_t qd = p[d] / s, rd = p[d] % s;
                lo[d] = int(rd == 0 ? qd - 1 : qd);
                hi[d] = int(qd);
            }
            bool edge = false;
            for (int ck = lo[2]; ck <= hi[2] && !edge; ++ck)
                for (int cj = lo[1]; cj <= hi[1] && !edge; ++cj)
                    for (int ci = lo[0]; ci <= hi[0] && !edge; ++ci)
                        if (ci >= 0 && cj >= 0 && ck >= 0 && ci < N && cj < N && ck < N && !cells.count(oct_key(l, ci, cj, ck)))
                            edge = true;
            if (edge) L.flags[t] = 2;
        });
        if (l > coarsest) {
            const OctLevelHost& C = o.levels[l - 1 - coarsest];
            L.parent.assign(L.nodes.size(), 0xFFFFFFFFu);
            L.pos.assign(L.nodes.size(), 0);
            for (size_t n = 0; n < L.cells.size(); ++n) {
                const uint64_t c = L.cells[n];
                const uint64_t par = parent_key(c);
                const auto it = std::lower_bound(C.cells.begin(), C.cells.end(), par);
                if (it == C.cells.end() || *it != par) return "level cell without parent";
                const uint32_t pi = uint32_t(it - C.cells.begin());
                const int off[3] = {oct_i(c) & 1, oct_j(c) & 1, oct_k(c) & 1};
                for (int a = 0; a < 27; ++a) {
                    const int32_t node = L.cell_nodes[n * 27 + a];
                    if (L.parent[node] != 0xFFFFFFFFu) continue;
                    const int loc[3] = {a % 3, (a / 3) % 3, a / 9};
                    L.parent[node] = pi;
                    L.pos[node] = uint16_t((2 * off[0] + loc[0]) + 5 * (2 * off[1] + loc[1]) + 25 * (2 * off[2] + loc[2]));
                }
            }
        }
    }
    // ---- copy indices: each active node to its coarsest leaf's level
    o.copy_index.resize(o.unodes.size());
    const char* err = parallel_check(o.unodes.size(), [&](size_t n) -> const char* {
        const int l = o.copy_level[n];
        const OctLevelHost& L = o.levels[l - coarsest];
        const auto it = std::lower_bound(L.nodes.begin(), L.nodes.end(), o.unodes[n]);
        if (it == L.nodes.end() || *it != o.unodes[n]) return "active node missing on its level";
        o.copy_index[n] = int32_t(it - L.nodes.begin());
        if (L.flags[o.copy_index[n]] == 2) return "active node on the refinement edge of its level";
        return nullptr;
    });
    if (err) return err;
    return "";
}

// Gradient indicator (Section 3.3: a gradient-based estimator refines about 1/7 of the cells per
// cycle; the estimator is not specified). Reading: eta_K = h^(5/2) |grad u_h(x_K)|_F, the Q2
// velocity's gradient at the leaf centre, where the basis reduces d/dx u to the difference of the
// two face-centre values over h (local nodes 12 and 14 along x, 10 and 16 along y, 4 and 22 along
// z). Leaf values come from the active vector through the hanging-node constraints; Dirichlet
// values are read as 0 (the wall condition), whatever the vector holds there.
void oct_gradient_indicator(const OctHost& o, const double* u, std::vector<double>& eta) {
    static const int kPairs[3][2] = {{12, 14}, {10, 16}, {4, 22}};
    const size_t nn = o.unodes.size(), nl = o.leaves.size();
    eta.assign(nl, 0.0);
    auto value = [&](int c, int32_t ref) {
        if (ref >= 0) return o.ubnd[size_t(ref)] ? 0.0 : u[size_t(c) * nn + size_t(ref)];
        const size_t h = size_t(-(ref + 1));
        double v = 0.0;
        for (int t = 0; t < kOctUCon; ++t) {
            const int32_t node = o.ucon_node[h * kOctUCon + t];
            if (node >= 0 && !o.ubnd[size_t(node)]) v += o.ucon_w[h * kOctUCon + t] * u[size_t(c) * nn + size_t(node)];
        }
        return v;
    };
    parallel_for(nl, [&](size_t n) {
        const double h = o.leaf_h[n];
        double sq = 0.0;
        for (int c = 0; c < 3; ++c)
            for (const auto& pr : kPairs) {
                const double d = (value(c, o.leaf_u[n * 27 + pr[1]]) - value(c, o.leaf_u[n * 27 + pr[0]])) / h;
                sq += d * d;
            }
        eta[n] = h * h * std::sqrt(h) * std::sqrt(sq);
    });
}

// Split the floor(n fraction + 1/2) leaves with the largest eta (equal eta: smaller key first),
// then 2:1 balance. `leaves` sorted, eta in the same order; returns the sorted new leaves.
std::vector<uint64_t> oct_refine_by_indicator(const std::vector<uint64_t>& leaves, const std::vector<double>& eta,
                                              double fraction) {
    const size_t n = leaves.size();
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    par_sort(order, [&](size_t a, size_t b) {   // a total order: keys are unique
        return eta[a] != eta[b] ? eta[a] > eta[b] : leaves[a] < leaves[b];
    });
    const size_t m = std::min(n, size_t(std::floor(double(n) * fraction + 0.5)));
    std::vector<uint8_t> mark(n, 0);
    for (size_t i = 0; i < m; ++i) mark[order[i]] = 1;
    std::vector<uint64_t> out;
    out.reserve(n + 7 * m);
    for (size_t i = 0; i < n; ++i) {
        if (!mark[i]) {
            out.push_back(leaves[i]);
            continue;
        }
        uint64_t ch[8];
        children_of(leaves[i], ch);
        out.insert(out.end(), ch, ch + 8);
    }
    return oct_balance(out);
}

}  // namespace stk
