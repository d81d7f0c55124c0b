"""The boundary is a C ABI: a plain C99 program that includes include/ers.h and links the
library calls its host-only entry points (no GPU): default options, the symbolic analysis
of a small pattern, and the solve/refactor plan check."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include "ers.h"

int main(void) {
  /* 4-node path graph with its diagonal: rows 0..3, columns sorted */
  int32_t rowptr[5] = {0, 2, 5, 8, 10};
  int32_t colidx[10] = {0, 1, 0, 1, 2, 1, 2, 3, 2, 3};
  double val[10] = {2, -1, -1, 2, -1, -1, 2, -1, -1, 2};
  ers_csr G = {4, 4, 10, rowptr, colidx, val};
  ers_opts o;
  ers_stats_t st;
  int32_t perm[4];
  int64_t counts[8];
  if (ers_default_opts(&o) != ERS_OK) return 1;
  if (ers_analyze(&G, &o, &st, perm) != ERS_OK) return 2;
  if (ers_solve_plan_check(&G, &o, counts) != ERS_OK) return 3;
  printf("%d %lld %lld %g %d\n", (int)st.n, (long long)st.nnz_L, (long long)counts[0],
         o.eps_krylov, (int)o.m_max);
  /* struct layouts, for the binding's mirror of them */
  printf("%zu %zu %zu %zu %zu %d\n", sizeof(ers_opts), offsetof(ers_opts, ordering),
         sizeof(ers_stats_t), offsetof(ers_stats_t, host_syncs), offsetof(ers_stats_t, host_polls),
         (int)o.ordering);
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib_dir():
    from paper_1511_04515_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_1511_04515_gb300")


def test_c_program_uses_the_library(lib_dir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    work = os.path.join(lib_dir, "_build", "c_abi")      # the package's (ignored) build folder
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "use_ers.c")
    exe = os.path.join(work, "use_ers")
    with open(src, "w") as f:
        f.write(PROGRAM)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), src, "-L", lib_dir, "-lers",
           f"-Wl,-rpath,{lib_dir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    line1, line2 = r.stdout.strip().splitlines()
    n, nnz_l, entries, eps, m_max = line1.split()
    assert int(n) == 4 and int(nnz_l) == 7          # a path has no fill: 4 + 3 entries
    assert int(entries) >= 1 and float(eps) == 1e-7 and int(m_max) == 40
    # the ctypes mirrors in the binding have the header's layout
    import ctypes
    from paper_1511_04515_gb300 import ers
    so, off_ord, ss, off_sync, off_poll, ordering = (int(v) for v in line2.split())
    assert so == ctypes.sizeof(ers.Opts) and off_ord == ers.Opts.ordering.offset
    assert ss == ctypes.sizeof(ers.Stats)
    assert off_sync == ers.Stats.host_syncs.offset and off_poll == ers.Stats.host_polls.offset
    assert ordering == ers.default_opts().ordering == 1
