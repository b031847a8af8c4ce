// Runs the autotuner's coordinate descent (paper_2506_01576_gb300/csrc/
// gi_descent.h) on synthetic cost models with known optima; prints one line per
// case, "name ok" or "name FAIL ...".  Test infrastructure; not part of the library.
#include <cstdio>
#include <map>

#include "gi_descent.h"

using gi::tune::Move;

namespace {

int failures = 0;

void check(bool ok, const char* name, const char* what) {
  std::printf("%s %s%s%s\n", name, ok ? "ok" : "FAIL ", ok ? "" : what, "");
  if (!ok) ++failures;
}

struct Model {
  std::array<int64_t, 11> v{};
  std::map<std::pair<int, int64_t>, bool> invalid;
  int timings = 0;
  int fail_at = -1;  // the timing that reports an error
};

template <class Cost>
int run(Model& md, const std::vector<std::vector<Move>>& groups, std::array<int64_t, 11>& cur,
        Cost cost, double* best, uint32_t* trials, uint32_t* passes) {
  auto set = [&](int o, int64_t x) {
    if (md.invalid.count({o, x})) return GI_ERR_INVALID;
    md.v[o] = x;
    return GI_OK;
  };
  auto time = [&](int* rc) {
    *rc = (md.timings++ == md.fail_at) ? GI_ERR_CUDA : GI_OK;
    return cost(md.v);
  };
  md.v = cur;
  const double start = cost(md.v);
  return gi::tune::descend(groups, cur, set, time, start, best, trials, passes);
}

std::vector<Move> sweep(int o, std::initializer_list<int64_t> xs) {
  std::vector<Move> g;
  for (int64_t x : xs) g.push_back(gi::tune::one(o, x));
  return g;
}

}  // namespace

int main() {
  // 1. separable: each knob has its own best value; found in one pass, confirmed in a second
  {
    Model md;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[1] = 1, cur[2] = 1, cur[4] = 256;
    auto cost = [](const std::array<int64_t, 11>& v) {
      return 10.0 + (v[1] - 4) * (v[1] - 4) + 2.0 * (v[2] - 2) * (v[2] - 2) + (v[4] == 512 ? 0.0 : 3.0);
    };
    std::vector<std::vector<Move>> g = {sweep(1, {1, 2, 4, 8}), sweep(2, {1, 2, 4}), sweep(4, {128, 256, 512})};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_OK && cur[1] == 4 && cur[2] == 2 && cur[4] == 512 && best == 10.0 && passes == 2,
          "separable", "optimum not reached");
    check(md.v == cur, "separable_applied", "the target was left at another setting");
  }
  // 2. a pair move: pinned levels help only together with a persistent grid
  {
    Model md;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[3] = 0, cur[5] = 0;
    auto cost = [](const std::array<int64_t, 11>& v) {
      if (v[3] > 0 && v[5] == 0) return 20.0;  // pinning without a persistent grid: slower
      if (v[3] == 0 && v[5] > 0) return 12.0;  // persistent grid alone: slower
      return v[3] > 0 ? 8.0 - v[3] : 10.0;
    };
    std::vector<Move> pin = sweep(3, {0, 1, 2});
    for (int64_t x : {1, 2})
      for (int64_t b : {1, 2}) pin.push_back(gi::tune::two(3, x, 5, b));
    std::vector<std::vector<Move>> g = {sweep(5, {0, 1, 2}), pin};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_OK && cur[3] == 2 && cur[5] > 0 && best == 6.0, "pair_move", "pair not found");
  }
  // 3. invalid values are skipped, never timed
  {
    Model md;
    md.invalid[{1, 8}] = true;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[1] = 1;
    auto cost = [](const std::array<int64_t, 11>& v) { return v[1] == 8 ? 1.0 : 10.0 - v[1]; };
    std::vector<std::vector<Move>> g = {sweep(1, {1, 2, 4, 8})};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_OK && cur[1] == 4 && best == 6.0, "invalid_skipped", "an invalid value was taken");
  }
  // 4. changes under 1% are not taken
  {
    Model md;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[4] = 256;
    auto cost = [](const std::array<int64_t, 11>& v) { return v[4] == 512 ? 99.5 : 100.0; };
    std::vector<std::vector<Move>> g = {sweep(4, {128, 256, 512})};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_OK && cur[4] == 256 && best == 100.0 && passes == 1, "threshold", "a <1% change was kept");
  }
  // 5. a timing error ends the search with that error
  {
    Model md;
    md.fail_at = 1;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[1] = 1;
    auto cost = [](const std::array<int64_t, 11>& v) { return 10.0 - v[1]; };
    std::vector<std::vector<Move>> g = {sweep(1, {1, 2, 4, 8})};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_ERR_CUDA, "error_propagates", "the error was lost");
  }
  // 6. at most 3 passes even when every pass changes something
  {
    Model md;
    std::array<int64_t, 11> cur;
    cur.fill(-1);
    cur[1] = 0, cur[2] = 0;
    // a staircase: each knob can only step one value past the other's
    auto cost = [](const std::array<int64_t, 11>& v) {
      if (v[1] > v[2] + 1 || v[2] > v[1]) return 1000.0;
      return 100.0 - 10.0 * (double)(v[1] + v[2]);
    };
    std::vector<std::vector<Move>> g = {sweep(1, {0, 1, 2, 3, 4, 5, 6, 7, 8}), sweep(2, {0, 1, 2, 3, 4, 5, 6, 7, 8})};
    double best = 0;
    uint32_t trials = 0, passes = 0;
    const int rc = run(md, g, cur, cost, &best, &trials, &passes);
    check(rc == GI_OK && passes == 3 && cur[1] == 3 && cur[2] == 3, "pass_limit", "pass limit not applied");
  }
  return failures ? 1 : 0;
}
