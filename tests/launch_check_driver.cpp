// Host driver of the debug build's launch checks (launch_check.h), compiled and run by
// tests/test_launch_check_cpu.py: prints "<case> <site>" for valid launches of every plan kind
// and for launches with one planted fault each.
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "launch_check.h"

using ptg::LaunchFacts;

static int padded_width(int nx) { return ((nx + 3 + 3) / 4) * 4; }

// the one-shot pass of a 128 x 128 grid, Nt = 1024 in 32 slices, on cluster launches
static LaunchFacts cluster128(int kind) {
  LaunchFacts f;
  f.kind = kind;
  f.Ntau = 32;
  f.M = 32;
  f.ny = 128;
  f.W = padded_width(128);
  f.cs = 16;
  f.rmax = 9;                     // 16 x 9 = 144 >= 129 node rows
  const bool sweep = kind == 2 || kind == 5;
  f.s0 = 0;
  f.ns = sweep ? 0 : 32;
  f.ntasks = sweep ? 1 : 32;
  f.has_hist = true;
  f.hist_j0 = 0;
  f.hist_rows = 1025;
  return f;
}

// a streamed launch of a 256 x 256 grid in 64 slices, with the multigrid hierarchy laid out as
// the library lays it out (six levels, 256 .. 8 elements a side)
static LaunchFacts streamed256(int kind) {
  LaunchFacts f;
  f.kind = kind;
  f.Ntau = 64;
  f.M = 32;
  f.ny = 256;
  f.W = padded_width(256);
  const bool sweep = kind == 2 || kind == 5;
  f.s0 = 0;
  f.ns = sweep ? 0 : 64;
  f.ntasks = sweep ? 1 : 64;
  f.has_hist = true;
  f.hist_rows = 2049;
  f.streamed = true;
  f.cs = sweep ? 128 : 2;
  f.rmax = (257 + f.cs - 1) / f.cs;
  f.groups = sweep ? 1 : 64;
  f.st_groups = 64;
  f.st_pv = (long long)(256 + 3) * f.W + 2 * 4;
  int n = 256, L = 0;
  long long voff = 0;
  while (true) {
    const long long plen = (long long)(n + 3) * padded_width(n) + 2 * 4;
    f.mg_voff[L] = voff;
    f.mg_plen[L] = plen;
    voff += (L == 0 ? 2 : 4) * plen;
    ++L;
    if (n % 2 != 0 || n <= 8 || L == ptg::kCheckMaxLevels) break;
    n /= 2;
  }
  f.mg_levels = L;
  f.mg_ws_stride = voff;
  return f;
}

int main() {
  struct Case {
    std::string name;
    std::function<LaunchFacts()> make;
  };
  std::vector<Case> cases = {
      {"ok_fine_primal", [] { return cluster128(0); }},
      {"ok_fine_chained",
       [] {
         LaunchFacts f = cluster128(0);
         f.chained = 1;
         f.ntasks = 1;
         return f;
       }},
      {"ok_coarse_adjoint", [] { return cluster128(4); }},
      {"ok_adjoint_sweep", [] { return cluster128(5); }},
      {"ok_adjoint_sweep_plt",
       [] {
         LaunchFacts f = cluster128(5);
         f.plt = 1;
         f.has_hist = false;
         f.hist_rows = 0;
         return f;
       }},
      {"ok_slice_range",
       [] {
         LaunchFacts f = cluster128(4);
         f.s0 = 8;
         f.ns = f.ntasks = 24;
         return f;
       }},
      {"ok_streamed_coarse", [] { return streamed256(1); }},
      {"ok_streamed_sweep", [] { return streamed256(5); }},
      {"slices_past_the_end",
       [] {
         LaunchFacts f = cluster128(0);
         f.s0 = 1;
         return f;
       }},
      {"slices_negative_start",
       [] {
         LaunchFacts f = cluster128(1);
         f.s0 = -1;
         f.ntasks = f.ns = 8;
         return f;
       }},
      {"chained_run_of_two_tasks",
       [] {
         LaunchFacts f = cluster128(3);
         f.chained = 1;
         f.ntasks = 2;
         return f;
       }},
      {"sweep_of_two_tasks",
       [] {
         LaunchFacts f = cluster128(2);
         f.ntasks = 2;
         return f;
       }},
      {"coarse_adjoint_without_history",
       [] {
         LaunchFacts f = cluster128(4);
         f.has_hist = false;
         return f;
       }},
      {"coarse_adjoint_history_short",
       [] {
         LaunchFacts f = cluster128(4);
         f.hist_rows = 32 * 31 + 1;   // the last slice reads row M (Ntau - 1) + 1
         return f;
       }},
      {"adjoint_sweep_history_offset",
       [] {
         LaunchFacts f = cluster128(5);
         f.hist_j0 = 1;
         return f;
       }},
      {"streamed_groups_over_workspace",
       [] {
         LaunchFacts f = streamed256(1);
         f.groups = 65;
         return f;
       }},
      {"streamed_sweep_two_groups",
       [] {
         LaunchFacts f = streamed256(2);
         f.groups = 2;
         return f;
       }},
      {"streamed_vector_too_short",
       [] {
         LaunchFacts f = streamed256(4);
         f.st_pv -= 1;
         return f;
       }},
      {"multigrid_workspace_short",
       [] {
         LaunchFacts f = streamed256(1);
         f.mg_ws_stride -= 1;
         return f;
       }},
      {"multigrid_too_many_levels",
       [] {
         LaunchFacts f = streamed256(1);
         f.mg_levels = ptg::kCheckMaxLevels + 1;
         return f;
       }},
      {"rows_not_covered",
       [] {
         LaunchFacts f = cluster128(0);
         f.rmax = 8;                  // 16 x 8 = 128 < 129 node rows
         return f;
       }},
      {"cluster_of_seventeen",
       [] {
         LaunchFacts f = cluster128(1);
         f.cs = 17;
         f.rmax = 8;
         return f;
       }},
  };
  for (const Case& c : cases) std::printf("%s %d\n", c.name.c_str(), ptg::launch_check_site(c.make()));
  return 0;
}
