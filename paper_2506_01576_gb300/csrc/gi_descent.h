// Coordinate descent over tuning knobs (the autotuner's search), host-only and
// independent of CUDA so that it can be tested on its own.
#pragma once

#include <stdint.h>

#include <array>
#include <vector>

#include "../../include/gi.h"

namespace gi {
namespace tune {

// ---------------------------------------------------------------- moves
// A move sets one knob, or two together (pinned levels only pay off with a
// persistent grid, Section 7.2, so those are tried as pairs).
struct Move {
  int n = 0;
  int opt[2] = {0, 0};
  int64_t val[2] = {0, 0};
};

inline Move one(int o, int64_t v) {
  Move m;
  m.n = 1;
  m.opt[0] = o;
  m.val[0] = v;
  return m;
}

inline Move two(int o0, int64_t v0, int o1, int64_t v1) {
  Move m;
  m.n = 2;
  m.opt[0] = o0;
  m.val[0] = v0;
  m.opt[1] = o1;
  m.val[1] = v1;
  return m;
}

// Coordinate descent over `groups` (one group per knob, its candidate moves).
// cur[o] holds the current value of option o (-1: not tuned); set(o, v) applies
// one value and returns GI_OK, or an error for a value the target rejects (that
// move is skipped); time(&rc) measures the current setting.  Each group keeps
// its fastest move if it beats the best time so far by at least 1%, the others
// held; passes over all groups repeat until one changes nothing, at most 3.
// Returns GI_OK, or the first error of time(); *best_out = the best time.
template <class Set, class Time>
int descend(const std::vector<std::vector<Move>>& groups, std::array<int64_t, 11>& cur, Set set,
            Time time, double start, double* best_out, uint32_t* trials, uint32_t* passes) {
  double best = start;
  for (int pass = 0; pass < 3; ++pass) {
    ++*passes;
    bool changed = false;
    for (const auto& group : groups) {
      std::array<int64_t, 11> keep = cur;
      for (const Move& mv : group) {
        bool same = true;
        for (int j = 0; j < mv.n; ++j) same &= cur[mv.opt[j]] == mv.val[j];
        if (same) continue;
        bool ok = true;
        for (int j = 0; j < mv.n && ok; ++j) ok = set(mv.opt[j], mv.val[j]) == GI_OK;
        if (ok) {
          int rc = GI_OK;
          const double t = time(&rc);
          if (rc != GI_OK) return rc;
          ++*trials;
          if (t < best * 0.99) {
            best = t;
            keep = cur;
            for (int j = 0; j < mv.n; ++j) keep[mv.opt[j]] = mv.val[j];
            changed = true;
          }
        }
        for (int j = 0; j < mv.n; ++j) set(mv.opt[j], cur[mv.opt[j]]);  // back to the current point
      }
      if (keep != cur) {
        cur = keep;
        for (int o = 1; o < 11; ++o)
          if (cur[o] >= 0) set(o, cur[o]);
      }
    }
    if (!changed) break;
  }
  *best_out = best;
  return GI_OK;
}

}  // namespace tune
}  // namespace gi
