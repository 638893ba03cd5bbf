// Portability tuning on the host: timing-table I/O, PortabilityTune (exact
// enumeration, greedy + swap), the library cost function, held-out scoring,
// and the manifest that carries the selected set to the runtime selector.
//
// Paper: Section IV-B (PortabilityTune returns a set kappa of variants for a
// set of inputs), Section IV-C (search over subsets of the variant space;
// its |inputs| * |K|^|kappa| cost), Section IV-D Eq. 1 (library cost
// function: geometric mean over environments of each environment's best
// performance relative to its Oracle), Section V-D (post-processing relative
// to the best variant per input), Fig. 1 (runtime inference).
#include <algorithm>
#include <array>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <limits>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "common.h"
#include "json.h"

namespace pt {

const char *kTableHeader =
    "shape_idx,M,N,K,transA,transB,variant,status,valid,median_ms,mean_ms,min_ms,reps,tflops,gbs,max_err";

bool same_shape(const pt_shape_t &a, const pt_shape_t &b) {
    return a.m == b.m && a.n == b.n && a.k == b.k && a.transA == b.transA && a.transB == b.transB;
}

std::string format_row(const TableRow &r) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%d,%lld,%lld,%lld,%c,%c,%s,%d,%d,%.9g,%.9g,%.9g,%d,%.6g,%.6g,%.6g",
                  r.shape_idx, (long long)r.shape.m, (long long)r.shape.n, (long long)r.shape.k, r.shape.transA,
                  r.shape.transB, r.variant.c_str(), r.status, r.valid, r.median_ms, r.mean_ms, r.min_ms, r.reps,
                  r.tflops, r.gbs, r.max_err);
    return buf;
}

static bool split_csv(const std::string &line, std::vector<std::string> *f) {
    f->clear();
    std::string cur;
    for (char c : line) {
        if (c == ',') {
            f->push_back(cur);
            cur.clear();
        } else if (c != '\r') {
            cur.push_back(c);
        }
    }
    f->push_back(cur);
    return true;
}

static bool to_ll(const std::string &s, long long *v) {
    if (s.empty()) return false;
    char *e = nullptr;
    errno = 0;
    *v = std::strtoll(s.c_str(), &e, 10);
    return errno == 0 && e && *e == 0;
}

static bool to_d(const std::string &s, double *v) {
    if (s.empty()) return false;
    char *e = nullptr;
    *v = std::strtod(s.c_str(), &e);
    return e && *e == 0;
}

int read_table(const char *path, Table *out) {
    std::ifstream in(path);
    if (!in) return set_error(PT_EIO, 1, "cannot open table '%s'", path);
    std::string line;
    if (!std::getline(in, line)) return set_error(PT_EFORMAT, 1, "empty table '%s'", path);
    if (!line.empty() && line.back() == '\r') line.pop_back();
    if (line != kTableHeader) return set_error(PT_EFORMAT, 1, "table '%s': unexpected header", path);
    Table t;
    std::map<std::string, int> vidx;
    std::vector<std::string> f;
    int lineno = 1;
    while (std::getline(in, line)) {
        ++lineno;
        if (line.empty() || line == "\r") continue;
        split_csv(line, &f);
        if (f.size() != 16) return set_error(PT_EFORMAT, 1, "table line %d: %zu fields", lineno, f.size());
        TableRow r;
        long long si, m, n, k, st, valid, reps;
        if (!to_ll(f[0], &si) || !to_ll(f[1], &m) || !to_ll(f[2], &n) || !to_ll(f[3], &k) || f[4].size() != 1 ||
            f[5].size() != 1 || f[6].empty() || !to_ll(f[7], &st) || !to_ll(f[8], &valid) ||
            !to_d(f[9], &r.median_ms) || !to_d(f[10], &r.mean_ms) || !to_d(f[11], &r.min_ms) ||
            !to_ll(f[12], &reps) || !to_d(f[13], &r.tflops) || !to_d(f[14], &r.gbs) || !to_d(f[15], &r.max_err))
            return set_error(PT_EFORMAT, 1, "table line %d: malformed field", lineno);
        if (m < 0 || n < 0 || k < 0 || (f[4][0] != 'N' && f[4][0] != 'T') || (f[5][0] != 'N' && f[5][0] != 'T') ||
            (valid != 0 && valid != 1))
            return set_error(PT_EFORMAT, 1, "table line %d: invalid value", lineno);
        if (valid && !(r.median_ms > 0 && std::isfinite(r.median_ms)))
            return set_error(PT_EFORMAT, 1, "table line %d: valid row without a positive time", lineno);
        r.shape_idx = (int)si;
        r.shape.m = m; r.shape.n = n; r.shape.k = k;
        r.shape.transA = f[4][0]; r.shape.transB = f[5][0];
        r.variant = f[6];
        r.status = (int)st; r.valid = (int)valid; r.reps = (int)reps;
        int s = -1;
        for (size_t i = 0; i < t.shapes.size(); ++i)
            if (same_shape(t.shapes[i], r.shape)) { s = (int)i; break; }
        if (s < 0) {
            s = (int)t.shapes.size();
            t.shapes.push_back(r.shape);
            for (auto &col : t.t) col.push_back(std::numeric_limits<double>::infinity());
        }
        auto it = vidx.find(r.variant);
        int v;
        if (it == vidx.end()) {
            v = (int)t.variants.size();
            vidx[r.variant] = v;
            t.variants.push_back(r.variant);
            t.t.emplace_back(t.shapes.size(), std::numeric_limits<double>::infinity());
        } else {
            v = it->second;
        }
        // A later row for the same (shape, variant) replaces an earlier one.
        t.t[v][s] = r.valid ? r.median_ms : std::numeric_limits<double>::infinity();
        t.rows.push_back(r);
    }
    *out = std::move(t);
    return PT_OK;
}

// ---- the cost function (Eq. 1, read as a performance to maximise) ---------------
namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct Problem {
    std::vector<int> cand;  // table variant indices, ascending registry id
    std::vector<int> reg;   // registry id of each candidate
    int S = 0;
    std::vector<double> lg;  // lg[c*S + s] = log(t_best[s] / t[cand[c]][s]), -inf if invalid
    double at(int c, int s) const { return lg[(size_t)c * S + s]; }
};

// t_best over every variant of the table.
std::vector<double> best_per_shape(const Table &t) {
    std::vector<double> b(t.shapes.size(), kInf);
    for (const auto &col : t.t)
        for (size_t s = 0; s < col.size(); ++s) b[s] = std::min(b[s], col[s]);
    return b;
}

int registry_id(const std::string &name) {
    const int id = pt_variant_by_name(name.c_str());
    return id;
}

int build_problem(const Table &t, const std::vector<int> &shapes, Problem *p) {
    const std::vector<double> tb = best_per_shape(t);
    std::vector<std::pair<int, int>> cands;  // (registry id, table index)
    for (size_t v = 0; v < t.variants.size(); ++v) {
        bool any = false;
        for (int s : shapes) any = any || std::isfinite(t.t[v][s]);
        if (!any) continue;
        const int id = registry_id(t.variants[v]);
        if (id < 0) return set_error(PT_EFORMAT, 1, "table variant '%s' is not in this library", t.variants[v].c_str());
        cands.emplace_back(id, (int)v);
    }
    std::sort(cands.begin(), cands.end());
    p->S = (int)shapes.size();
    p->cand.clear();
    p->reg.clear();
    for (auto &c : cands) {
        p->reg.push_back(c.first);
        p->cand.push_back(c.second);
    }
    p->lg.assign(p->cand.size() * (size_t)p->S, -kInf);
    for (size_t c = 0; c < p->cand.size(); ++c)
        for (int j = 0; j < p->S; ++j) {
            const double tv = t.t[p->cand[c]][shapes[j]];
            if (std::isfinite(tv)) p->lg[c * p->S + j] = std::log(tb[shapes[j]] / tv);
        }
    return PT_OK;
}

// Geomean of per-shape best-of-set performance given the per-shape max log.
double geomean_from(const std::vector<double> &mx, int S) {
    if (S == 0) return 1.0;
    double total = 0;
    for (int s = 0; s < S; ++s) {
        if (!std::isfinite(mx[s])) return 0.0;
        total += mx[s];
    }
    return std::exp(total / S);
}

double set_value(const Problem &p, const std::vector<int> &set) {
    std::vector<double> mx(p.S, -kInf);
    for (int c : set)
        for (int s = 0; s < p.S; ++s) mx[s] = std::max(mx[s], p.at(c, s));
    return geomean_from(mx, p.S);
}

// Exhaustive PortabilityTune: every k-subset of the candidates in
// lexicographic order; a later subset replaces the best only when strictly
// better, so exact ties keep the lexicographically smallest set.
void exact_rec(const Problem &p, int k, int start, std::vector<int> &cur, std::vector<std::vector<double>> &mx,
               std::vector<int> &best, double &best_val) {
    const int d = (int)cur.size();
    const int n = (int)p.cand.size();
    for (int c = start; c <= n - (k - d); ++c) {
        std::vector<double> &m = mx[d + 1];
        for (int s = 0; s < p.S; ++s) m[s] = std::max(mx[d][s], p.at(c, s));
        cur.push_back(c);
        if (d + 1 == k) {
            const double v = geomean_from(m, p.S);
            if (v > best_val) {
                best_val = v;
                best = cur;
            }
        } else {
            exact_rec(p, k, c + 1, cur, mx, best, best_val);
        }
        cur.pop_back();
    }
}

void select_exact(const Problem &p, int k, std::vector<int> *out, double *val) {
    const int n = (int)p.cand.size();
    if (k >= n) {
        out->resize(n);
        for (int i = 0; i < n; ++i) (*out)[i] = i;
        *val = set_value(p, *out);
        return;
    }
    std::vector<std::vector<double>> mx(k + 1, std::vector<double>(p.S, -kInf));
    std::vector<int> cur, best;
    double best_val = -1.0;
    exact_rec(p, k, 0, cur, mx, best, best_val);
    *out = best;
    *val = best_val;
}

// Greedy growth and 1-swap local search on the facility-location form
// F(kappa) = sum_s max_{v in kappa} max(lg[v][s], floor), which equals
// S * log(Eq. 1 value) whenever every shape is covered.
constexpr double kFloor = -30.0;

double f_value(const Problem &p, const std::vector<int> &set) {
    double tot = 0;
    for (int s = 0; s < p.S; ++s) {
        double m = kFloor;
        for (int c : set) m = std::max(m, p.at(c, s));
        tot += m;
    }
    return tot;
}

void local_search(const Problem &p, std::vector<int> &set) {
    const int n = (int)p.cand.size();
    const int k = (int)set.size();
    std::vector<char> in(n, 0);
    for (int c : set) in[c] = 1;
    while (true) {
        // Per shape: best and second-best member values and the best's slot.
        std::vector<double> b1(p.S, kFloor), b2(p.S, kFloor);
        std::vector<int> who(p.S, -1);
        for (int slot = 0; slot < k; ++slot)
            for (int s = 0; s < p.S; ++s) {
                const double v = std::max(p.at(set[slot], s), kFloor);
                if (v > b1[s]) { b2[s] = b1[s]; b1[s] = v; who[s] = slot; }
                else if (v > b2[s]) b2[s] = v;
            }
        double base = 0;
        for (int s = 0; s < p.S; ++s) base += b1[s];
        double best_gain = 1e-12;
        int best_slot = -1, best_c = -1;
        for (int slot = 0; slot < k; ++slot) {
            for (int c = 0; c < n; ++c) {
                if (in[c]) continue;
                double tot = 0;
                for (int s = 0; s < p.S; ++s) {
                    const double rest = (who[s] == slot) ? b2[s] : b1[s];
                    tot += std::max(rest, std::max(p.at(c, s), kFloor));
                }
                if (tot - base > best_gain) {
                    best_gain = tot - base;
                    best_slot = slot;
                    best_c = c;
                }
            }
        }
        if (best_slot < 0) break;
        in[set[best_slot]] = 0;
        in[best_c] = 1;
        set[best_slot] = best_c;
    }
    std::sort(set.begin(), set.end());
}

uint64_t splitmix(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void select_greedy_swap(const Problem &p, int k, uint64_t seed, std::vector<int> *out, double *val) {
    const int n = (int)p.cand.size();
    if (k >= n) {
        select_exact(p, k, out, val);
        return;
    }
    std::vector<int> best;
    double best_g = -1, best_f = -kInf;
    const int restarts = 8;
    uint64_t draw = 0;
    for (int r = 0; r < restarts; ++r) {
        std::vector<int> set;
        if (r == 0) {
            std::vector<char> in(n, 0);
            for (int step = 0; step < k; ++step) {
                int arg = -1;
                double bv = -kInf;
                for (int c = 0; c < n; ++c) {
                    if (in[c]) continue;
                    set.push_back(c);
                    const double f = f_value(p, set);
                    set.pop_back();
                    if (f > bv + 1e-12) { bv = f; arg = c; }
                }
                in[arg] = 1;
                set.push_back(arg);
            }
        } else {
            std::vector<char> in(n, 0);
            while ((int)set.size() < k) {
                const int c = (int)(splitmix(seed, draw++) % (uint64_t)n);
                if (!in[c]) { in[c] = 1; set.push_back(c); }
            }
        }
        local_search(p, set);
        const double g = set_value(p, set), f = f_value(p, set);
        if (g > best_g || (g == best_g && f > best_f) || (g == best_g && f == best_f && set < best)) {
            best_g = g;
            best_f = f;
            best = set;
        }
    }
    *out = best;
    *val = best_g;
}

double log_binom(int n, int k) { return std::lgamma(n + 1.0) - std::lgamma(k + 1.0) - std::lgamma(n - k + 1.0); }

// ---- alternative selections (Section IV-C) ------------------------------------------
// Points: the training shapes' performance vectors over the candidates,
// perf = t_best / t (0 where invalid).
std::vector<std::vector<double>> perf_points(const Table &t, const std::vector<int> &shapes, const Problem &p) {
    const std::vector<double> tb = best_per_shape(t);
    std::vector<std::vector<double>> pts(shapes.size(), std::vector<double>(p.cand.size(), 0.0));
    for (size_t j = 0; j < shapes.size(); ++j)
        for (size_t c = 0; c < p.cand.size(); ++c) {
            const double tv = t.t[p.cand[c]][shapes[j]];
            if (std::isfinite(tv)) pts[j][c] = tb[shapes[j]] / tv;
        }
    return pts;
}

double sqdist(const std::vector<double> &a, const std::vector<double> &b) {
    double d = 0.0;
    for (size_t i = 0; i < a.size(); ++i) d += (a[i] - b[i]) * (a[i] - b[i]);
    return d;
}

int argmax_first(const std::vector<double> &v) {
    int best = 0;
    for (int i = 1; i < (int)v.size(); ++i)
        if (v[i] > v[best]) best = i;
    return best;
}

double splitmix_u(uint64_t seed, uint64_t i) { return (double)(splitmix(seed, i) >> 11) * 0x1.0p-53; }

// k-means (Section IV-C-2): k-means++ initialisation with SplitMix64 draws,
// Lloyd iterations (nearest centroid, ties to the lower; an empty cluster
// keeps its centroid) until no assignment changes or 100 rounds; each
// centroid contributes its highest-performing candidate.
void select_kmeans(const Table &t, const std::vector<int> &shapes, const Problem &p, int k, uint64_t seed,
                   std::vector<int> *out) {
    const std::vector<std::vector<double>> pts = perf_points(t, shapes, p);
    const int n = (int)pts.size();
    if (k > n) k = n;
    uint64_t draws = 0;
    std::vector<int> chosen;
    std::vector<std::vector<double>> centers;
    const int first = (int)(splitmix_u(seed, draws++) * n);
    chosen.push_back(first);
    centers.push_back(pts[first]);
    while ((int)centers.size() < k) {
        std::vector<double> d2(n);
        double total = 0.0;
        for (int i = 0; i < n; ++i) {
            double m = sqdist(pts[i], centers[0]);
            for (size_t c = 1; c < centers.size(); ++c) m = std::min(m, sqdist(pts[i], centers[c]));
            d2[i] = m;
        }
        for (int i = 0; i < n; ++i) total += d2[i];
        int nxt = n - 1;
        if (total <= 0.0) {
            for (int i = 0; i < n; ++i)
                if (std::find(chosen.begin(), chosen.end(), i) == chosen.end()) {
                    nxt = i;
                    break;
                }
        } else {
            const double u = splitmix_u(seed, draws) * total;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                acc += d2[i];
                if (acc > u) {
                    nxt = i;
                    break;
                }
            }
        }
        ++draws;
        chosen.push_back(nxt);
        centers.push_back(pts[nxt]);
    }
    std::vector<int> assign(n, -1);
    for (int iter = 0; iter < 100; ++iter) {
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            int best = 0;
            double bd = sqdist(pts[i], centers[0]);
            for (int c = 1; c < (int)centers.size(); ++c) {
                const double d = sqdist(pts[i], centers[c]);
                if (d < bd) {
                    best = c;
                    bd = d;
                }
            }
            if (assign[i] != best) {
                assign[i] = best;
                changed = true;
            }
        }
        if (!changed) break;
        for (int c = 0; c < (int)centers.size(); ++c) {
            std::vector<double> mean(p.cand.size(), 0.0);
            int cnt = 0;
            for (int i = 0; i < n; ++i)
                if (assign[i] == c) {
                    for (size_t v = 0; v < mean.size(); ++v) mean[v] += pts[i][v];
                    ++cnt;
                }
            if (cnt) {
                for (double &x : mean) x /= cnt;
                centers[c] = mean;
            }
        }
    }
    out->clear();
    for (const auto &c : centers) {
        const int v = argmax_first(c);
        if (std::find(out->begin(), out->end(), v) == out->end()) out->push_back(v);
    }
    std::sort(out->begin(), out->end());
}

// Regression tree (Section IV-C-3) from (log2 M, log2 N, log2 K) to the
// performance vector, squared error summed over the vector, grown best-first
// to k leaves (ties: lower feature, lower threshold, earlier leaf); each leaf
// contributes the highest-performing candidate of its mean.
struct TreeNode {
    int feature = -1;
    double threshold = 0;
    int left = -1, right = -1;
    int variant = -1;  // leaves: registry id
};

void select_tree(const Table &t, const std::vector<int> &shapes, const Problem &p, int k, std::vector<int> *out,
                 std::vector<TreeNode> *tree) {
    const std::vector<std::vector<double>> pts = perf_points(t, shapes, p);
    const int n = (int)pts.size();
    const size_t dim = p.cand.size();
    std::vector<std::array<double, 3>> feats(n);
    for (int j = 0; j < n; ++j) {
        const pt_shape_t &sh = t.shapes[shapes[j]];
        feats[j] = {std::log2((double)sh.m), std::log2((double)sh.n), std::log2((double)sh.k)};
    }
    auto sum_of = [&](const std::vector<int> &idx) {
        std::vector<double> m(dim, 0.0);
        for (int i : idx)
            for (size_t v = 0; v < dim; ++v) m[v] += pts[i][v];
        return m;
    };
    auto sse = [&](const std::vector<int> &idx) {
        if (idx.empty()) return 0.0;
        std::vector<double> mean = sum_of(idx);
        for (double &x : mean) x /= (double)idx.size();
        double e = 0.0;
        for (int i : idx) e += sqdist(pts[i], mean);
        return e;
    };
    struct Split {
        bool ok = false;
        double gain = 0, thr = 0;
        int f = -1;
        std::vector<int> left, right;
    };
    auto best_split = [&](const std::vector<int> &idx) {
        Split best;
        const double base = sse(idx);
        for (int f = 0; f < 3; ++f) {
            std::vector<double> vals;
            for (int i : idx) vals.push_back(feats[i][f]);
            std::sort(vals.begin(), vals.end());
            vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
            for (size_t q = 0; q + 1 < vals.size(); ++q) {
                const double thr = 0.5 * (vals[q] + vals[q + 1]);
                std::vector<int> l, r;
                for (int i : idx) (feats[i][f] <= thr ? l : r).push_back(i);
                const double gain = base - sse(l) - sse(r);
                if (!best.ok || gain > best.gain) {
                    best.ok = true;
                    best.gain = gain;
                    best.f = f;
                    best.thr = thr;
                    best.left = l;
                    best.right = r;
                }
            }
        }
        return best;
    };
    std::vector<std::vector<int>> leaves(1);
    for (int i = 0; i < n; ++i) leaves[0].push_back(i);
    std::vector<int> leaf_node(1, 0);
    tree->assign(1, TreeNode());
    while ((int)leaves.size() < k) {
        Split cand;
        int cli = -1;
        for (int li = 0; li < (int)leaves.size(); ++li) {
            Split b = best_split(leaves[li]);
            if (b.ok && b.gain > 0.0 && (cli < 0 || b.gain > cand.gain)) {
                cand = b;
                cli = li;
            }
        }
        if (cli < 0) break;
        const int node = leaf_node[cli];
        const int ln = (int)tree->size(), rn = ln + 1;
        tree->push_back(TreeNode());
        tree->push_back(TreeNode());
        (*tree)[node].feature = cand.f;
        (*tree)[node].threshold = cand.thr;
        (*tree)[node].left = ln;
        (*tree)[node].right = rn;
        leaves[cli] = cand.left;
        leaves.insert(leaves.begin() + cli + 1, cand.right);
        leaf_node[cli] = ln;
        leaf_node.insert(leaf_node.begin() + cli + 1, rn);
    }
    out->clear();
    for (size_t li = 0; li < leaves.size(); ++li) {
        const int c = argmax_first(sum_of(leaves[li]));
        (*tree)[leaf_node[li]].variant = p.reg[c];
        if (std::find(out->begin(), out->end(), c) == out->end()) out->push_back(c);
    }
    std::sort(out->begin(), out->end());
}

}  // namespace

// ---- time model of the runtime selector -----------------------------------------------
void model_features(const pt_shape_t &s, double f[kModelFeatures]) {
    const double u = (std::log2((double)s.m) - 9.0) / 3.0, v = (std::log2((double)s.n) - 9.0) / 3.0,
                 w = (std::log2((double)s.k) - 9.0) / 3.0;
    const double x[kModelFeatures] = {1.0, u, v, w, u * u, v * v, w * w, u * v, u * w, v * w};
    for (int i = 0; i < kModelFeatures; ++i) f[i] = x[i];
}

// Least squares min |X c - y| over the first p columns of X (n rows) by
// Householder QR; false when the columns are numerically dependent
// (|R_ii| <= 1e-9 max_j |R_jj|).
static bool lstsq_qr(std::vector<std::vector<double>> X, std::vector<double> y, int p, std::vector<double> *c) {
    const int n = (int)X.size();
    if (n < p) return false;
    std::vector<double> diag(p);
    for (int j = 0; j < p; ++j) {
        double norm = 0;
        for (int i = j; i < n; ++i) norm += X[i][j] * X[i][j];
        norm = std::sqrt(norm);
        if (norm == 0) return false;
        const double alpha = X[j][j] > 0 ? -norm : norm;
        std::vector<double> vv(n, 0.0);
        vv[j] = X[j][j] - alpha;
        for (int i = j + 1; i < n; ++i) vv[i] = X[i][j];
        double vn = 0;
        for (int i = j; i < n; ++i) vn += vv[i] * vv[i];
        if (vn > 0) {
            for (int col = j; col < p; ++col) {
                double d = 0;
                for (int i = j; i < n; ++i) d += vv[i] * X[i][col];
                d = 2 * d / vn;
                for (int i = j; i < n; ++i) X[i][col] -= d * vv[i];
            }
            double d = 0;
            for (int i = j; i < n; ++i) d += vv[i] * y[i];
            d = 2 * d / vn;
            for (int i = j; i < n; ++i) y[i] -= d * vv[i];
        }
        diag[j] = X[j][j];
    }
    double mx = 0;
    for (int j = 0; j < p; ++j) mx = std::max(mx, std::fabs(diag[j]));
    for (int j = 0; j < p; ++j)
        if (std::fabs(diag[j]) <= 1e-9 * mx) return false;
    c->assign(kModelFeatures, 0.0);
    for (int j = p - 1; j >= 0; --j) {
        double sacc = y[j];
        for (int col = j + 1; col < p; ++col) sacc -= X[j][col] * (*c)[col];
        (*c)[j] = sacc / X[j][j];
    }
    return true;
}

// Coefficients for one member from its valid training times: the quadratic
// model when it is determined (>= 10 points, independent features), else the
// linear one (>= 4), else the mean; empty when no training time is valid.
static std::vector<double> fit_member(const std::vector<pt_shape_t> &shapes, const std::vector<double> &times) {
    std::vector<std::vector<double>> X;
    std::vector<double> y;
    for (size_t j = 0; j < shapes.size(); ++j) {
        if (!std::isfinite(times[j]) || times[j] <= 0) continue;
        std::vector<double> f(kModelFeatures);
        model_features(shapes[j], f.data());
        X.push_back(f);
        y.push_back(std::log(times[j]));
    }
    std::vector<double> c;
    if (X.empty()) return c;
    for (int p : {kModelFeatures, 4})
        if ((int)X.size() >= p && lstsq_qr(X, y, p, &c)) return c;
    c.assign(kModelFeatures, 0.0);
    double sum = 0;
    for (double v : y) sum += v;
    c[0] = sum / (double)y.size();
    return c;
}

// ln t - model at every training shape (NaN where the member is invalid);
// empty when the member has no model.
static std::vector<double> member_residuals(const std::vector<double> &coef, const std::vector<pt_shape_t> &shapes,
                                            const std::vector<double> &times) {
    std::vector<double> r;
    if (coef.empty()) return r;
    for (size_t j = 0; j < shapes.size(); ++j) {
        if (!std::isfinite(times[j]) || times[j] <= 0) {
            r.push_back(std::nan(""));
            continue;
        }
        double f[kModelFeatures];
        model_features(shapes[j], f);
        double pred = 0;
        for (int i = 0; i < kModelFeatures; ++i) pred += coef[i] * f[i];
        r.push_back(std::log(times[j]) - pred);
    }
    return r;
}

// L1 distance of two shapes in (log2 M, log2 N, log2 K).
static double log_distance(const pt_shape_t &a, const pt_shape_t &b) {
    return std::fabs(std::log2((double)a.m) - std::log2((double)b.m)) +
           std::fabs(std::log2((double)a.n) - std::log2((double)b.n)) +
           std::fabs(std::log2((double)a.k) - std::log2((double)b.k));
}

// ---- manifest --------------------------------------------------------------------
static std::string shape_json(const pt_shape_t &s) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "\"m\": %lld, \"n\": %lld, \"k\": %lld, \"transA\": \"%c\", \"transB\": \"%c\"",
                  (long long)s.m, (long long)s.n, (long long)s.k, s.transA, s.transB);
    return buf;
}

static int write_manifest(const char *path, const char *method, int k, double g, const std::vector<int> &kappa_ids,
                          const std::vector<std::pair<pt_shape_t, int>> &map, const std::vector<TreeNode> *tree,
                          const std::vector<std::vector<double>> *coef, char ta, char tb,
                          const std::vector<pt_shape_t> *pts, const std::vector<std::vector<double>> *resid) {
    std::ofstream o(path);
    if (!o) return set_error(PT_EIO, 9, "cannot write manifest '%s'", path);
    auto name = [](int id) {
        pt_variant_desc_t d;
        pt_variant_desc(id, &d);
        return std::string(d.name);
    };
    char gbuf[64];
    std::snprintf(gbuf, sizeof(gbuf), "%.17g", g);
    o << "{\n  \"format\": \"pt-manifest-1\",\n  \"method\": " << json::quote(method) << ",\n  \"k\": " << k
      << ",\n  \"train_geomean\": " << gbuf << ",\n  \"kappa\": [";
    for (size_t i = 0; i < kappa_ids.size(); ++i) o << (i ? ", " : "") << json::quote(name(kappa_ids[i]));
    o << "],\n  \"map\": [";
    for (size_t i = 0; i < map.size(); ++i)
        o << (i ? ",\n" : "\n") << "    {" << shape_json(map[i].first)
          << ", \"variant\": " << json::quote(name(map[i].second)) << "}";
    o << "\n  ]";
    if (tree && !tree->empty()) {
        // Regression tree over (log2 M, log2 N, log2 K); node 0 is the root.
        o << ",\n  \"tree\": [";
        for (size_t i = 0; i < tree->size(); ++i) {
            const TreeNode &nd = (*tree)[i];
            char buf[128];
            if (nd.feature >= 0)
                std::snprintf(buf, sizeof(buf), "{\"feature\": %d, \"threshold\": %.17g, \"left\": %d, \"right\": %d}",
                              nd.feature, nd.threshold, nd.left, nd.right);
            o << (i ? ",\n" : "\n") << "    " << (nd.feature >= 0 ? std::string(buf)
                                                           : "{\"variant\": " + json::quote(name(nd.variant)) + "}");
        }
        o << "\n  ]";
    }
    if (coef && !coef->empty()) {
        // Time model (see model_features), one coefficient list per kappa member.
        o << ",\n  \"model\": {\"transA\": \"" << ta << "\", \"transB\": \"" << tb
          << "\", \"features\": \"1,u,v,w,u2,v2,w2,uv,uw,vw; u = (log2 M - 9) / 3\", \"coef\": [";
        for (size_t i = 0; i < coef->size(); ++i) {
            o << (i ? ",\n" : "\n") << "    ";
            if ((*coef)[i].empty()) {
                o << "null";
                continue;
            }
            o << "[";
            for (int f = 0; f < kModelFeatures; ++f) {
                char buf[40];
                std::snprintf(buf, sizeof(buf), "%.17g", (*coef)[i][f]);
                o << (f ? ", " : "") << buf;
            }
            o << "]";
        }
        o << "\n  ]";
        if (pts && resid && resid->size() == coef->size()) {
            // Residual correction: the training shapes and each member's
            // ln t - model at them (null where it is invalid).
            o << ",\n  \"points\": [";
            for (size_t j = 0; j < pts->size(); ++j)
                o << (j ? ", " : "") << "[" << (long long)(*pts)[j].m << ", " << (long long)(*pts)[j].n << ", "
                  << (long long)(*pts)[j].k << "]";
            o << "],\n  \"resid\": [";
            for (size_t i = 0; i < resid->size(); ++i) {
                o << (i ? ",\n" : "\n") << "    ";
                if ((*resid)[i].empty()) {
                    o << "null";
                    continue;
                }
                o << "[";
                for (size_t j = 0; j < (*resid)[i].size(); ++j) {
                    char buf[40];
                    if (std::isfinite((*resid)[i][j]))
                        std::snprintf(buf, sizeof(buf), "%.17g", (*resid)[i][j]);
                    else
                        std::snprintf(buf, sizeof(buf), "null");
                    o << (j ? ", " : "") << buf;
                }
                o << "]";
            }
            o << "\n  ]";
        }
        o << "}";
    }
    o << "\n}\n";
    o.flush();
    if (!o) return set_error(PT_EIO, 9, "write failed for '%s'", path);
    return PT_OK;
}

int read_manifest(const char *path, Manifest *out) {
    std::ifstream in(path);
    if (!in) return set_error(PT_EIO, 1, "cannot open manifest '%s'", path);
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string text = ss.str();
    json::Value root;
    json::Parser parser(text);
    if (!parser.parse(&root) || root.kind != json::Value::Object)
        return set_error(PT_EFORMAT, 1, "manifest '%s': not a JSON object", path);
    const json::Value *fmt = root.get("format");
    if (!fmt || fmt->kind != json::Value::String || fmt->str != "pt-manifest-1")
        return set_error(PT_EFORMAT, 1, "manifest '%s': unknown format", path);
    Manifest m;
    if (const json::Value *me = root.get("method"); me && me->kind == json::Value::String) m.method = me->str;
    if (const json::Value *g = root.get("train_geomean"); g && g->kind == json::Value::Number) m.train_geomean = g->num;
    const json::Value *kap = root.get("kappa");
    if (!kap || kap->kind != json::Value::Array || kap->arr.empty())
        return set_error(PT_EFORMAT, 1, "manifest '%s': kappa missing or empty", path);
    for (const auto &v : kap->arr) {
        if (v.kind != json::Value::String) return set_error(PT_EFORMAT, 1, "manifest: kappa entry is not a name");
        const int id = pt_variant_by_name(v.str.c_str());
        if (id < 0) return set_error(PT_EFORMAT, 1, "manifest: unknown variant '%s'", v.str.c_str());
        m.kappa.push_back(id);
    }
    const json::Value *map = root.get("map");
    if (map) {
        if (map->kind != json::Value::Array) return set_error(PT_EFORMAT, 1, "manifest: map is not an array");
        for (const auto &e : map->arr) {
            const json::Value *vm = e.get("m"), *vn = e.get("n"), *vk = e.get("k"), *ta = e.get("transA"),
                              *tb = e.get("transB"), *var = e.get("variant");
            if (!vm || !vn || !vk || !ta || !tb || !var || vm->kind != json::Value::Number ||
                vn->kind != json::Value::Number || vk->kind != json::Value::Number ||
                ta->kind != json::Value::String || tb->kind != json::Value::String ||
                var->kind != json::Value::String || ta->str.size() != 1 || tb->str.size() != 1 || vm->num < 1 ||
                vn->num < 1 || vk->num < 1)
                return set_error(PT_EFORMAT, 1, "manifest: malformed map entry");
            ManifestEntry me;
            me.shape.m = (int64_t)vm->num;
            me.shape.n = (int64_t)vn->num;
            me.shape.k = (int64_t)vk->num;
            me.shape.transA = ta->str[0];
            me.shape.transB = tb->str[0];
            me.variant = pt_variant_by_name(var->str.c_str());
            if (me.variant < 0) return set_error(PT_EFORMAT, 1, "manifest: unknown variant '%s'", var->str.c_str());
            if (std::find(m.kappa.begin(), m.kappa.end(), me.variant) == m.kappa.end())
                return set_error(PT_EFORMAT, 1, "manifest: map names a variant outside kappa");
            m.map.push_back(me);
        }
    }
    if (const json::Value *tr = root.get("tree"); tr) {
        if (tr->kind != json::Value::Array) return set_error(PT_EFORMAT, 1, "manifest: tree is not an array");
        const int nn = (int)tr->arr.size();
        for (const auto &e : tr->arr) {
            ManifestNode nd;
            if (const json::Value *v = e.get("variant"); v) {
                if (v->kind != json::Value::String) return set_error(PT_EFORMAT, 1, "manifest: bad tree leaf");
                nd.variant = pt_variant_by_name(v->str.c_str());
                if (nd.variant < 0) return set_error(PT_EFORMAT, 1, "manifest: unknown variant '%s'", v->str.c_str());
            } else {
                const json::Value *f = e.get("feature"), *th = e.get("threshold"), *l = e.get("left"),
                                  *r = e.get("right");
                if (!f || !th || !l || !r || f->kind != json::Value::Number || th->kind != json::Value::Number ||
                    l->kind != json::Value::Number || r->kind != json::Value::Number || f->num < 0 || f->num > 2 ||
                    l->num < 1 || l->num >= nn || r->num < 1 || r->num >= nn)
                    return set_error(PT_EFORMAT, 1, "manifest: bad tree node");
                nd.feature = (int)f->num;
                nd.threshold = th->num;
                nd.left = (int)l->num;
                nd.right = (int)r->num;
            }
            m.tree.push_back(nd);
        }
        // Children must come after their parent (no cycles).
        for (int i = 0; i < nn; ++i)
            if (m.tree[i].feature >= 0 && (m.tree[i].left <= i || m.tree[i].right <= i))
                return set_error(PT_EFORMAT, 1, "manifest: tree nodes out of order");
    }
    if (const json::Value *md = root.get("model"); md) {
        const json::Value *ta = md->get("transA"), *tb = md->get("transB"), *cf = md->get("coef");
        if (!ta || !tb || !cf || ta->kind != json::Value::String || tb->kind != json::Value::String ||
            ta->str.size() != 1 || tb->str.size() != 1 || cf->kind != json::Value::Array ||
            cf->arr.size() != m.kappa.size())
            return set_error(PT_EFORMAT, 1, "manifest: malformed model");
        m.model_ta = ta->str[0];
        m.model_tb = tb->str[0];
        for (const auto &e : cf->arr) {
            std::vector<double> c;
            if (e.kind == json::Value::Array) {
                if (e.arr.size() != (size_t)kModelFeatures) return set_error(PT_EFORMAT, 1, "manifest: bad model row");
                for (const auto &x : e.arr) {
                    if (x.kind != json::Value::Number || !std::isfinite(x.num))
                        return set_error(PT_EFORMAT, 1, "manifest: bad model coefficient");
                    c.push_back(x.num);
                }
            } else if (e.kind != json::Value::Null) {
                return set_error(PT_EFORMAT, 1, "manifest: bad model row");
            }
            m.coef.push_back(std::move(c));
        }
        const json::Value *pv = md->get("points"), *rv = md->get("resid");
        if (pv || rv) {
            if (!pv || !rv || pv->kind != json::Value::Array || rv->kind != json::Value::Array ||
                rv->arr.size() != m.kappa.size())
                return set_error(PT_EFORMAT, 1, "manifest: malformed model residuals");
            for (const auto &e : pv->arr) {
                if (e.kind != json::Value::Array || e.arr.size() != 3)
                    return set_error(PT_EFORMAT, 1, "manifest: bad model point");
                double d[3];
                for (int q = 0; q < 3; ++q) {
                    if (e.arr[q].kind != json::Value::Number || !(e.arr[q].num >= 1))
                        return set_error(PT_EFORMAT, 1, "manifest: bad model point");
                    d[q] = e.arr[q].num;
                }
                pt_shape_t sh;
                sh.m = (int64_t)d[0];
                sh.n = (int64_t)d[1];
                sh.k = (int64_t)d[2];
                sh.transA = m.model_ta;
                sh.transB = m.model_tb;
                m.model_pts.push_back(sh);
                m.model_pts_log2.push_back(std::log2((double)sh.m));
                m.model_pts_log2.push_back(std::log2((double)sh.n));
                m.model_pts_log2.push_back(std::log2((double)sh.k));
            }
            for (size_t i = 0; i < rv->arr.size(); ++i) {
                const json::Value &e = rv->arr[i];
                std::vector<double> r;
                if (e.kind == json::Value::Array) {
                    if (e.arr.size() != m.model_pts.size() || m.coef[i].empty())
                        return set_error(PT_EFORMAT, 1, "manifest: bad residual row");
                    for (const auto &x : e.arr) {
                        if (x.kind == json::Value::Null) {
                            r.push_back(std::nan(""));
                        } else if (x.kind == json::Value::Number && std::isfinite(x.num)) {
                            r.push_back(x.num);
                        } else {
                            return set_error(PT_EFORMAT, 1, "manifest: bad residual");
                        }
                    }
                } else if (e.kind != json::Value::Null) {
                    return set_error(PT_EFORMAT, 1, "manifest: bad residual row");
                }
                m.resid.push_back(std::move(r));
            }
        }
    }
    *out = std::move(m);
    return PT_OK;
}

// Runtime selector (Fig. 1 inference step): exact hit; else the tree (tree
// manifests); else the time model (the member with the smallest predicted
// time, ties to the earlier member; shapes with the model's transposes);
// else the nearest listed shape with the same transposes (any transposes if
// none) in log2 space, L1 distance, ties to the earlier entry; with no map,
// the first member.
int manifest_pick(const Manifest &m, const pt_shape_t &s) {
    if (m.kappa.empty()) return -1;
    if (m.map.empty()) return m.kappa[0];
    for (const auto &e : m.map)
        if (same_shape(e.shape, s)) return e.variant;
    if (!m.tree.empty()) {
        const double f[3] = {std::log2((double)s.m), std::log2((double)s.n), std::log2((double)s.k)};
        int node = 0;
        for (size_t steps = 0; steps <= m.tree.size() && m.tree[node].feature >= 0; ++steps)
            node = f[m.tree[node].feature] <= m.tree[node].threshold ? m.tree[node].left : m.tree[node].right;
        if (m.tree[node].variant >= 0) return m.tree[node].variant;
    }
    if (!m.coef.empty() && s.transA == m.model_ta && s.transB == m.model_tb) {
        double f[kModelFeatures];
        model_features(s, f);
        // Distances from the query to the model's points, once per pick: the
        // same L1 distance in (log2 M, log2 N, log2 K) for every member.
        const size_t np = m.model_pts.size();
        std::vector<double> dist(np);
        const double q[3] = {std::log2((double)s.m), std::log2((double)s.n), std::log2((double)s.k)};
        const bool have_logs = m.model_pts_log2.size() == 3 * np;
        for (size_t j = 0; j < np; ++j)
            dist[j] = have_logs ? std::fabs(q[0] - m.model_pts_log2[3 * j]) + std::fabs(q[1] - m.model_pts_log2[3 * j + 1]) +
                                      std::fabs(q[2] - m.model_pts_log2[3 * j + 2])
                                : log_distance(s, m.model_pts[j]);
        int best = -1;
        double bp = kInf;
        for (size_t i = 0; i < m.kappa.size() && i < m.coef.size(); ++i) {
            if (m.coef[i].empty()) continue;
            double pred = 0;
            for (int j = 0; j < kModelFeatures; ++j) pred += m.coef[i][j] * f[j];
            if (i < m.resid.size() && !m.resid[i].empty()) {
                // Residual correction: 1/d^2-weighted mean of the member's
                // residuals at its valid training shapes; at distance 0 the
                // mean of those shapes' residuals (their measured ln t).
                double num = 0, den = 0, at = 0;
                int n_at = 0;
                for (size_t j = 0; j < np; ++j) {
                    const double r = m.resid[i][j];
                    if (!std::isfinite(r)) continue;
                    const double d = dist[j];
                    if (d == 0.0) {
                        at += r;
                        ++n_at;
                    } else {
                        num += r / (d * d);
                        den += 1.0 / (d * d);
                    }
                }
                if (n_at > 0)
                    pred += at / n_at;
                else if (den > 0)
                    pred += num / den;
            }
            if (pred < bp) {
                bp = pred;
                best = m.kappa[i];
            }
        }
        if (best >= 0) return best;
    }
    bool any_same_trans = false;
    for (const auto &e : m.map)
        any_same_trans = any_same_trans || (e.shape.transA == s.transA && e.shape.transB == s.transB);
    const double q[3] = {std::log2((double)s.m), std::log2((double)s.n), std::log2((double)s.k)};
    int best = -1;
    double best_d = kInf;
    for (const auto &e : m.map) {
        if (any_same_trans && (e.shape.transA != s.transA || e.shape.transB != s.transB)) continue;
        const double d = std::fabs(std::log2((double)e.shape.m) - q[0]) + std::fabs(std::log2((double)e.shape.n) - q[1]) +
                         std::fabs(std::log2((double)e.shape.k) - q[2]);
        if (d < best_d) {
            best_d = d;
            best = e.variant;
        }
    }
    return best;
}

}  // namespace pt

using namespace pt;

extern "C" {

int pt_table_shapes(const char *table_path, int *out_n) {
    clear_error();
    if (!table_path) return set_error(PT_EINVAL, 1, "table_path is NULL");
    if (!out_n) return set_error(PT_EINVAL, 2, "out_n is NULL");
    Table t;
    int rc = read_table(table_path, &t);
    if (rc != PT_OK) return rc;
    *out_n = (int)t.shapes.size();
    return PT_OK;
}

int pt_table_shape(const char *table_path, int i, pt_shape_t *out) {
    clear_error();
    if (!table_path) return set_error(PT_EINVAL, 1, "table_path is NULL");
    if (!out) return set_error(PT_EINVAL, 3, "out is NULL");
    Table t;
    int rc = read_table(table_path, &t);
    if (rc != PT_OK) return rc;
    if (i < 0 || i >= (int)t.shapes.size()) return set_error(PT_EINVAL, 2, "shape index out of range");
    *out = t.shapes[i];
    return PT_OK;
}

int pt_select(const char *table_path, const int *train_idx, int n_train, int k, int method, uint64_t seed,
              int *out_ids, double *out_train_geomean, const char *manifest_path) {
    clear_error();
    if (!table_path) return set_error(PT_EINVAL, 1, "table_path is NULL");
    if (k < 1) return set_error(PT_EINVAL, 4, "k must be >= 1");
    if (n_train < 0 || (n_train > 0 && !train_idx)) return set_error(PT_EINVAL, 2, "bad training list");
    if (!out_ids) return set_error(PT_EINVAL, 7, "out_ids is NULL");
    Table t;
    int rc = read_table(table_path, &t);
    if (rc != PT_OK) return rc;
    std::vector<int> shapes;
    if (n_train == 0) {
        for (size_t s = 0; s < t.shapes.size(); ++s) shapes.push_back((int)s);
    } else {
        for (int i = 0; i < n_train; ++i) {
            if (train_idx[i] < 0 || train_idx[i] >= (int)t.shapes.size())
                return set_error(PT_EINVAL, 2, "training shape index %d out of range", train_idx[i]);
            shapes.push_back(train_idx[i]);
        }
    }
    if (shapes.empty()) return set_error(PT_EINVAL, 2, "no training shapes");
    Problem p;
    rc = build_problem(t, shapes, &p);
    if (rc != PT_OK) return rc;
    if (p.cand.empty()) return set_error(PT_EFORMAT, 1, "no variant is valid on the training shapes");
    std::vector<int> set;
    std::vector<TreeNode> tree;
    double val = 0;
    const char *mname = "exact";
    switch (method) {
        case PT_SELECT_EXACT:
            if (k < (int)p.cand.size() && log_binom((int)p.cand.size(), k) > std::log(5e8))
                return set_error(PT_EUNSUPPORTED, 5, "exact enumeration of C(%zu,%d) subsets is too large",
                                 p.cand.size(), k);
            select_exact(p, k, &set, &val);
            break;
        case PT_SELECT_GREEDY_SWAP:
            mname = "greedy_swap";
            select_greedy_swap(p, k, seed, &set, &val);
            break;
        case PT_SELECT_AUTO:
            if (k >= (int)p.cand.size() || log_binom((int)p.cand.size(), k) <= std::log(2e7)) {
                select_exact(p, k, &set, &val);
            } else {
                mname = "greedy_swap";
                select_greedy_swap(p, k, seed, &set, &val);
            }
            break;
        case PT_SELECT_KMEANS:
            mname = "kmeans";
            select_kmeans(t, shapes, p, k, seed, &set);
            val = set_value(p, set);
            break;
        case PT_SELECT_TREE:
            mname = "tree";
            select_tree(t, shapes, p, k, &set, &tree);
            val = set_value(p, set);
            break;
        default:
            return set_error(PT_EINVAL, 5, "unknown selection method %d", method);
    }
    std::vector<int> ids;
    for (int c : set) ids.push_back(p.reg[c]);
    for (int i = 0; i < k; ++i) out_ids[i] = i < (int)ids.size() ? ids[i] : -1;
    if (out_train_geomean) *out_train_geomean = val;
    if (manifest_path) {
        // Shape map: each training shape's fastest member (ties -> lowest id).
        std::vector<std::pair<pt_shape_t, int>> map;
        for (int j = 0; j < p.S; ++j) {
            int best = -1;
            double bt = kInf;
            for (int c : set) {
                const double tv = t.t[p.cand[c]][shapes[j]];
                if (tv < bt) {
                    bt = tv;
                    best = p.reg[c];
                }
            }
            if (best >= 0) map.emplace_back(t.shapes[shapes[j]], best);
        }
        // Time model over the training shapes, when they share one transpose pair.
        std::vector<std::vector<double>> coef, resid;
        std::vector<pt_shape_t> tr;
        bool one_pair = true;
        for (int j = 1; j < p.S; ++j)
            one_pair = one_pair && t.shapes[shapes[j]].transA == t.shapes[shapes[0]].transA &&
                       t.shapes[shapes[j]].transB == t.shapes[shapes[0]].transB;
        if (one_pair) {
            for (int j = 0; j < p.S; ++j) tr.push_back(t.shapes[shapes[j]]);
            for (int c : set) {
                std::vector<double> tv;
                for (int j = 0; j < p.S; ++j) tv.push_back(t.t[p.cand[c]][shapes[j]]);
                coef.push_back(fit_member(tr, tv));
                resid.push_back(member_residuals(coef.back(), tr, tv));
            }
        }
        rc = write_manifest(manifest_path, mname, k, val, ids, map, method == PT_SELECT_TREE ? &tree : nullptr,
                            one_pair ? &coef : nullptr, t.shapes[shapes[0]].transA, t.shapes[shapes[0]].transB,
                            one_pair ? &tr : nullptr, one_pair ? &resid : nullptr);
        if (rc != PT_OK) return rc;
    }
    return PT_OK;
}

int pt_score(const char *table_path, const int *ids, int k, const int *shape_idx, int n, int mode,
             const char *manifest_path, double *out_geomean) {
    clear_error();
    if (!table_path) return set_error(PT_EINVAL, 1, "table_path is NULL");
    if (!out_geomean) return set_error(PT_EINVAL, 8, "out_geomean is NULL");
    if (n < 0 || (n > 0 && !shape_idx)) return set_error(PT_EINVAL, 4, "bad shape list");
    Table t;
    int rc = read_table(table_path, &t);
    if (rc != PT_OK) return rc;
    std::map<int, int> reg_to_table;
    for (size_t v = 0; v < t.variants.size(); ++v) {
        const int id = pt_variant_by_name(t.variants[v].c_str());
        if (id >= 0) reg_to_table[id] = (int)v;
    }
    clear_error();
    auto time_of = [&](int id, int s) {
        auto it = reg_to_table.find(id);
        return it == reg_to_table.end() ? kInf : t.t[it->second][s];
    };
    const std::vector<double> tb = best_per_shape(t);
    std::vector<int> shapes;
    for (int i = 0; i < n; ++i) {
        if (shape_idx[i] < 0 || shape_idx[i] >= (int)t.shapes.size())
            return set_error(PT_EINVAL, 4, "shape index %d out of range", shape_idx[i]);
        shapes.push_back(shape_idx[i]);
    }
    double total = 0;
    if (mode == PT_SCORE_BEST_OF_SET) {
        if (k < 1 || !ids) return set_error(PT_EINVAL, 2, "bad id list");
        for (int s : shapes) {
            double m = kInf;
            for (int i = 0; i < k; ++i)
                if (ids[i] >= 0) m = std::min(m, time_of(ids[i], s));
            if (!std::isfinite(m)) {
                *out_geomean = 0.0;
                return PT_OK;
            }
            total += std::log(tb[s] / m);
        }
    } else if (mode == PT_SCORE_SELECTOR) {
        if (!manifest_path) return set_error(PT_EINVAL, 7, "selector scoring needs a manifest");
        Manifest m;
        rc = read_manifest(manifest_path, &m);
        if (rc != PT_OK) return rc;
        for (int s : shapes) {
            const int pick = manifest_pick(m, t.shapes[s]);
            double tv = time_of(pick, s);
            // Same fallback order as pt_sgemm: other members, then the default.
            for (size_t i = 0; !std::isfinite(tv) && i < m.kappa.size(); ++i) tv = time_of(m.kappa[i], s);
            if (!std::isfinite(tv)) tv = time_of(0, s);
            if (!std::isfinite(tv)) {
                *out_geomean = 0.0;
                return PT_OK;
            }
            total += std::log(tb[s] / tv);
        }
    } else {
        return set_error(PT_EINVAL, 6, "unknown scoring mode %d", mode);
    }
    *out_geomean = shapes.empty() ? 1.0 : std::exp(total / shapes.size());
    return PT_OK;
}

}  // extern "C"
