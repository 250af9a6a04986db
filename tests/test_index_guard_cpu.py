"""Index arithmetic of the lattice Boltzmann kernels, on the CPU.

The neighbourhood (Hood) and the index guard of the checked build (chk) are
host-callable.  A small host program, compiled by nvcc from the library's own
headers, walks every node of lattices from 1 x 1 x 1 up to several tiles. For
each node it compares every x + c_i and x - c_i that the kernels form with the
index of the wrapped coordinates: periodic across a periodic face, clamped to
the edge node across a mirror or wall face (Sec. II.B's stencils at a
symmetry plane).  Compiled with -DDSM_CHECKED it also checks that chk latches
the bounds bit and clamps to 0, and that no in-range index sets the bit; in the
normal build chk is the identity.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_19941_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "dsm_lb_impl.cuh"
using namespace dsm;

static int wrap(int v, int n, int lo_face, int hi_face) {
  if (v < 0) return lo_face ? 0 : n - 1;
  if (v >= n) return hi_face ? n - 1 : 0;
  return v;
}

template <class L>
static long long walk(int nx, int ny, int nz, const int (&face)[6], int *err, int *bad) {
  long long count = 0;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        Hood h;
        h.init_faces(x, y, z, nx, ny, nz, face);
        h.guard(err);
        const int n = h.g(h.ox[1] + h.oy[1] + h.oz[1]);
        if (n != x + nx * (y + ny * z)) (*bad)++;
        for (int i = 0; i < L::Q; i++) {
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            const int px = wrap(x + sgn * L::cx(i), nx, face[0], face[1]);
            const int py = wrap(y + sgn * L::cy(i), ny, face[2], face[3]);
            const int pz = wrap(z + sgn * L::cz(i), nz, face[4], face[5]);
            const int want = px + nx * (py + ny * pz);
            const int got = sgn > 0 ? h.template plus<L>(i) : h.template minus<L>(i);
            if (got != want) (*bad)++;
            if (sgn > 0 && h.template plus_rt<L>(i) != want) (*bad)++;
            count += 2;
          }
        }
      }
  return count;
}

int main() {
  int bad = 0, err = 0;
  long long count = 0;
  const int shapes3[][3] = {{1, 1, 1}, {3, 1, 1}, {1, 5, 2}, {5, 4, 3}, {7, 5, 3}, {33, 9, 4}};
  const int shapes2[][2] = {{1, 1}, {3, 1}, {1, 5}, {5, 4}, {23, 17}, {64, 9}};
  for (int fm = 0; fm < 64; fm++) {
    int face[6];
    for (int k = 0; k < 6; k++) face[k] = (fm >> k) & 1 ? 1 + (k & 1) : 0;  // mirror or wall
    for (auto &s : shapes3) count += walk<Lat<1>>(s[0], s[1], s[2], face, &err, &bad);
    int face2[6] = {face[0], face[1], face[2], face[3], 0, 0};
    for (auto &s : shapes2) count += walk<Lat<0>>(s[0], s[1], 1, face2, &err, &bad);
  }
  if (err) { std::printf("in-range index latched %d\n", err); return 3; }
  if (bad) { std::printf("%d wrong neighbour indices\n", bad); return 2; }
  int e = 0;
#ifdef DSM_CHECKED
  const bool ok = chk(&e, 9, 10) == 9 && e == 0 && chk(&e, 10, 10) == 0 && (e & ERR_BOUNDS) &&
                  (e = 0, chk(&e, -1, 10) == 0) && (e & ERR_BOUNDS) &&
                  (e = 0, chk(&e, 4LL << 32, 4LL << 32) == 0) && (e & ERR_BOUNDS) &&
                  chk((int *)nullptr, 11, 10) == 0;
  const char *build = "checked";
#else
  const bool ok = chk(&e, 10, 10) == 10 && chk(&e, -1, 10) == -1 && e == 0;
  const char *build = "normal";
#endif
  if (!ok) { std::printf("chk misbehaves (%s build)\n", build); return 4; }
  std::printf("ok %lld indices (%s build)\n", count, build);
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not available")


@pytest.mark.parametrize("checked", [False, True])
def test_neighbour_indices_and_guard(tmp_path, checked):
    src = tmp_path / "hood.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "hood"
    cmd = [_nvcc(), "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
           "arch=compute_103a,code=sm_103a", "-I", CSRC, str(src), "-o", str(exe)]
    if checked:
        cmd.insert(1, "-DDSM_CHECKED")
    subprocess.run(cmd, check=True, capture_output=True, text=True, timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
    assert ("checked" if checked else "normal") in r.stdout
