// launch_check.h -- the launch checks of the debug build (-DPTG_DEBUG, libptg_debug.so).  Before
// every launch of an op's task kinds the index ranges the launch will touch are compared with
// what the op allocated; a failed check skips the launch and reports PTG_EBOUNDS with the site
// below (ptg_stats.fail_kind = 30 + task kind, fail_step = site) instead of letting a kernel
// read or write out of bounds.  Plain host C++ with no CUDA types, so that it compiles on its
// own for the CPU tests.
#pragma once

namespace ptg {

constexpr int kCheckMaxLevels = 10;   // multigrid levels of a launch at most
constexpr int kCheckSlack = 4;        // entries before and after a padded array (kSlack)

enum LaunchSite : int {
  kSiteNone = 0,
  kSiteSlices = 1,      // fine and coarse kinds: the launch's slices lie in [0, Ntau) (a chained
                        // run is one task); a correction sweep is one task
  kSiteHistory = 2,     // rows read from the history by absolute time index lie in its window:
                        // G_adj of slice s reads M s + 1 and M s + 1 - M (clamped at 0), the
                        // adjoint sweep M s + 1 of every slice; the window starts at row 0
  kSiteGroups = 3,      // streamed launches: at most the op's workspace groups (a sweep runs
                        // in its own group: one group)
  kSiteWorkspace = 4,   // a streamed group's vectors hold the padded node layout with its slack
  kSiteMgLevels = 5,    // every multigrid level's vectors lie inside a group's workspace
  kSiteRows = 6,        // the CTAs of a task own every node row between them, and a cluster
                        // launch has at most 16 CTAs per cluster
};

// What a launch will touch and what the op holds (task kinds as in ptg_internal.h: 0 fine
// primal, 1 coarse primal, 2 primal sweep, 3 fine adjoint, 4 coarse adjoint, 5 adjoint sweep).
struct LaunchFacts {
  int kind = 0;
  int s0 = 0, ns = 0, chained = 0, ntasks = 0;
  int Ntau = 0, M = 0;
  int plt = 0;                         // correction kinds with G = 0 (no history read)
  bool has_hist = false;
  int hist_j0 = 0, hist_rows = 0;
  int ny = 0, W = 0;                   // element rows and padded row width of the op's grid
  int cs = 0, rmax = 0;                // CTAs per task (cluster or group) and most rows per CTA
  bool streamed = false, wide = false;
  int groups = 0;                      // streamed: groups launched
  int st_groups = 0;                   // streamed: the op's workspace groups (the sweeps' group
                                       // comes after them)
  long long st_pv = 0;                 // streamed: entries of one vector, slack included
  int mg_levels = 0;
  long long mg_voff[kCheckMaxLevels] = {};
  long long mg_plen[kCheckMaxLevels] = {};
  long long mg_ws_stride = 0;          // floats of one group's multigrid workspace
};

// The first failed check, or kSiteNone.
inline int launch_check_site(const LaunchFacts& f) {
  const bool sweep = f.kind == 2 || f.kind == 5;
  if (sweep) {
    if (f.ntasks != 1) return kSiteSlices;
  } else {
    const int n = f.chained ? f.ns : f.ntasks;
    if (f.s0 < 0 || n < 1 || f.s0 + n > f.Ntau || (f.chained && f.ntasks != 1)) return kSiteSlices;
  }
  long long need = -1;                 // highest history row read by absolute index
  if (f.kind == 4) need = (long long)f.M * (f.s0 + f.ntasks - 1) + 1;
  if (f.kind == 5 && !f.plt) need = (long long)f.M * (f.Ntau - 1) + 1;
  if (need >= 0 && (!f.has_hist || f.hist_j0 != 0 || need >= f.hist_rows)) return kSiteHistory;
  if (f.streamed) {
    if (f.groups < 1 || (sweep ? f.groups != 1 : f.groups > f.st_groups)) return kSiteGroups;
    if (f.st_pv < (long long)(f.ny + 3) * f.W + 2 * kCheckSlack) return kSiteWorkspace;
    if (f.mg_levels < 0 || f.mg_levels > kCheckMaxLevels) return kSiteMgLevels;
    for (int l = 0; l < f.mg_levels; ++l) {
      const long long vecs = l == 0 ? 2 : 4;   // level 0: u, res; coarser: f, u, res, e
      if (f.mg_voff[l] < 0 || f.mg_plen[l] <= 0 || f.mg_voff[l] + vecs * f.mg_plen[l] > f.mg_ws_stride)
        return kSiteMgLevels;
    }
  }
  if (f.cs < 1 || f.rmax < 1 || (long long)f.cs * f.rmax < f.ny + 1) return kSiteRows;
  if (!f.streamed && !f.wide && f.cs > 16) return kSiteRows;
  return kSiteNone;
}

}  // namespace ptg
