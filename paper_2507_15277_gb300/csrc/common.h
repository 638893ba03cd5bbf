// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pt_sgemm.h"

namespace pt {

int set_error(int code, int arg, const char *fmt, ...);
void clear_error();
bool verbose();

// ---- timing table --------------------------------------------------------------
struct TableRow {
    int shape_idx = -1;
    pt_shape_t shape{};
    std::string variant;  // name (stable key)
    int status = 0;       // PT_OK or the launch status
    int valid = 0;
    double median_ms = 0, mean_ms = 0, min_ms = 0;
    int reps = 0;
    double tflops = 0, gbs = 0, max_err = 0;
};

struct Table {
    std::vector<pt_shape_t> shapes;      // distinct shapes, first-appearance order
    std::vector<std::string> variants;   // distinct variant names, first-appearance order
    std::vector<std::vector<double>> t;  // t[v][s] median ms, +inf when invalid / missing
    std::vector<TableRow> rows;
};

int read_table(const char *path, Table *out);
extern const char *kTableHeader;
std::string format_row(const TableRow &r);
bool same_shape(const pt_shape_t &a, const pt_shape_t &b);

// ---- manifest (the multi-versioned set and its shape map) ----------------------
struct ManifestEntry {
    pt_shape_t shape;
    int variant;  // registry id
};

// Node of a regression-tree selector: internal nodes test feature
// (0: log2 M, 1: log2 N, 2: log2 K) <= threshold; leaves name a variant.
struct ManifestNode {
    int feature = -1;
    double threshold = 0;
    int left = -1, right = -1;
    int variant = -1;
};

// Time model of the runtime selector: per kappa member, ln(median ms) as a
// quadratic in u = (log2 M - 9) / 3, v = (log2 N - 9) / 3, w = (log2 K - 9) / 3
// with features [1, u, v, w, u^2, v^2, w^2, uv, uw, vw], least-squares fitted
// on the training shapes (fewer terms when the member has too few valid
// training shapes, none when it has none).
constexpr int kModelFeatures = 10;
void model_features(const pt_shape_t &s, double f[kModelFeatures]);

struct Manifest {
    std::string method;
    std::vector<int> kappa;  // registry ids, in manifest order
    std::vector<ManifestEntry> map;
    std::vector<ManifestNode> tree;  // optional; shapes outside the map descend it
    // Optional time model: coef[i] for kappa[i] (empty: no model for it);
    // applies to shapes with transposes (model_ta, model_tb).
    std::vector<std::vector<double>> coef;
    char model_ta = 0, model_tb = 0;
    // Optional residual correction of the model: the training shapes
    // (model_pts) and, per member, ln t - model at each of them (resid[i][j];
    // NaN where the member is invalid; resid[i] empty: no correction).  The
    // prediction at an unlisted shape adds the 1/d^2-weighted mean of the
    // member's residuals, d the L1 distance in (log2 M, log2 N, log2 K).
    std::vector<pt_shape_t> model_pts;
    std::vector<double> model_pts_log2;  // (log2 M, log2 N, log2 K) of each point, 3 per point
    std::vector<std::vector<double>> resid;
    double train_geomean = 0;
};

int read_manifest(const char *path, Manifest *out);
// The runtime selector's pick for a shape (-1 if the manifest is empty).
int manifest_pick(const Manifest &m, const pt_shape_t &s);
// Installed manifest (copy under the library mutex).
bool installed_manifest(Manifest *out);

}  // namespace pt
