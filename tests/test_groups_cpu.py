"""Host logic of the grouped FP64 evaluation (static_ops.h), compiled with
g++ and checked on the CPU: which compile-time table terms form groups (the
star / heat family's six axial neighbours; the climate operator's three
biharmonic rings of four and its vertical pair; nothing for the 2D 5-point
operator, whose sweeps must stay bit-identical to the fused 2D kernel), and
the weight test that decides whether a plan takes the group evaluation."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1207_1746_b300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstring>
#include "static_ops.h"
using namespace gscl;
template <class Def> void groups(const char *name) {
  std::printf("%s axial %d coef", name, axial_group<Def>());
  for (int i = 0; i < Def::NT; ++i)
    if (coef_group_start<Def>(i) == i) std::printf(" %d:%d", i, coef_group_len<Def>(i));
  std::printf(" any %d\n", (int)has_groups<Def>());
}
int main() {
  groups<OpHeat7Rhs>("heat7rhs");
  groups<OpStar7>("star7");
  groups<OpJacobi7Rhs>("jacobi7rhs");
  groups<OpJacobi5_2D>("jacobi5_2d");
  groups<OpHeat7Fused>("heat7fused");
  groups<OpClimate>("climate");
  // climate weights in table order (dt = dz = 1): per output the unit term,
  // the biharmonic (-20, 8 x4, -2 x4, -1 x4), the vertical pair (-1/2, +1/2),
  // the tendency
  double w[51];
  for (int m = 0; m < 3; ++m) {
    double *p = w + 17 * m;
    p[0] = 1.0; p[1] = -20.0;
    for (int k = 0; k < 4; ++k) { p[2 + k] = 8.0; p[6 + k] = -2.0; p[10 + k] = -1.0; }
    p[14] = -0.5; p[15] = 0.5; p[16] = 1.0;
  }
  std::printf("climate_ok %d\n", (int)static_group_weights_ok(OP_CLIMATE, w));
  w[17 + 7] = std::nextafter(-2.0, 0.0);
  std::printf("climate_ring_off %d\n", (int)static_group_weights_ok(OP_CLIMATE, w));
  w[17 + 7] = -2.0; w[34 + 15] = -0.5;
  std::printf("climate_pair_same_sign %d\n", (int)static_group_weights_ok(OP_CLIMATE, w));
  double h[8] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
  std::printf("heat_ok %d\n", (int)static_group_weights_ok(OP_HEAT7_RHS, h));
  h[4] = -0.125;
  std::printf("heat_sign_off %d\n", (int)static_group_weights_ok(OP_HEAT7_RHS, h));
  double j[4] = {0.25, 0.25, 0.25, 0.25};
  std::printf("jacobi5_ok %d\n", (int)static_group_weights_ok(OP_JACOBI5_2D, j));
  return 0;
}
"""


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("groups")
    (d / "h.cpp").write_text(HARNESS)
    exe = d / "h"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-include", "cmath", "-I", CSRC, "-o", str(exe),
                           str(d / "h.cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {line.split()[0]: line.split(None, 1)[1] for line in out.splitlines()}


def test_star_family_has_the_axial_group(report):
    # the unit offsets follow the centre term (heat, star) or come first (Jacobi, fused)
    assert report["heat7rhs"] == "axial 1 coef any 1"
    assert report["star7"] == "axial 1 coef any 1"
    assert report["jacobi7rhs"] == "axial 0 coef any 1"
    assert report["heat7fused"] == "axial 0 coef any 1"


def test_two_dimensional_five_point_operator_has_no_group(report):
    assert report["jacobi5_2d"] == "axial -1 coef any 0"


def test_climate_groups_are_its_rings_and_vertical_pairs(report):
    # per output m (17 terms from 17 m): rings of four at 2, 6, 10, the pair at 14
    want = " ".join(f"{17 * m + k}:{n}" for m in range(3) for k, n in ((2, 4), (6, 4), (10, 4), (14, 2)))
    assert report["climate"] == f"axial -1 coef {want} any 1"


def test_weight_test(report):
    assert report["climate_ok"] == "1"
    assert report["climate_ring_off"] == "0"        # one ring weight one ulp off
    assert report["climate_pair_same_sign"] == "0"  # a pair must be opposite
    assert report["heat_ok"] == "1"
    assert report["heat_sign_off"] == "0"
    assert report["jacobi5_ok"] == "0"              # no group: table order
