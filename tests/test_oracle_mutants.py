"""The oracles' pins catch plausible mistakes (CPU).

Each case plants one mistake -- a dropped term, a wrong sign, a swapped operand or
index -- in a temporary copy of an oracle and runs the pins named for it against that
copy.  For the C++ oracle (oracle/nimbus_oracle.cpp) the copy is built and loaded
through NIMBUS_ORACLE_LIB by tests/test_oracle_pins.py; for the labelling oracle
(oracle/segment.py) tests/test_segment_oracle.py runs in a temporary copy of the
repository's Python sources with the planted module.  A case passes when at least one
of those pins fails and none crashes.  The planted text must occur exactly once in
the source, so a change to an oracle that removes it shows up here rather than
silently weakening the check.  Nothing here touches the CUDA library or the committed
oracle build.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nimbus_oracle.cpp")
TINY = "test_image_method_room_tiny and not paper and not facing"

# (name, text in the oracle, planted mistake, pins expected to catch it (pytest -k))
MUTANTS = [
    ("eq1_weight_square_dropped",      # Eq. 1: Gaussian of the distance, not its square
     "double w = std::exp(-dot(d, d) * inv_s2);\n    sw += w;\n    sp = sp + w * P;",
     "double w = std::exp(-std::sqrt(dot(d, d)) * inv_s2);\n    sw += w;\n    sp = sp + w * P;",
     "two_points"),
    ("newton_placement_dropped",       # Section 2.2.1: hit placed at the last march point
     "double th = std::fabs(dn) > 1e-3 ? t - f / dn : t;", "double th = t;", "sdf_on_exact_plane"),
    ("sdf_segment_halved",             # Section 2.2.1: march over half a subvoxel diameter
     "  const double L = s.hs * std::sqrt(3.0);\n  double tc = dot(ie.bbc - P, d);",
     "  const double L = 0.5 * s.hs * std::sqrt(3.0);\n  double tc = dot(ie.bbc - P, d);", "subvoxel_diameter"),
    ("voxel_sphere_halved",            # Section 2.2.4: voxel spheres of half their radius
     "voxel_center(s, u[0], u[1], u[2]), s.r_vox))", "voxel_center(s, u[0], u[1], u[2]), 0.5 * s.r_vox))",
     "reflection_and_diffraction"),
    ("ie_sphere_halved",               # Section 2.2.4: entity spheres of half their radius
     "if (!cone_sphere(cone.apex, cone.axis, cone.sin_a, cone.cos_a, ie.sc, s.r_sub)) continue;",
     "if (!cone_sphere(cone.apex, cone.axis, cone.sin_a, cone.cos_a, ie.sc, 0.5 * s.r_sub)) continue;",
     "reflection_and_diffraction"),
    ("march_skip_adjacent",            # Section 2.2.4: no evaluation next to occupied voxels
     "if (ctx.march[cell_of(s, v[0], v[1], v[2])] > 1) return true;",
     "if (ctx.march[cell_of(s, v[0], v[1], v[2])] > 0) return true;", TINY),
    ("neighbourhood_reevaluated",      # a cone evaluating one neighbourhood twice
     "          if (have_last && std::abs(u[0] - last[0]) <= 1", "          if (false && have_last && std::abs(u[0] - last[0]) <= 1",
     "leaving"),
    ("keller_fan_half_count",          # Section 2.2.4: half the fan's cones
     "int M = (int)std::ceil(PI / alpha);", "int M = (int)std::ceil(PI / (2.0 * alpha));", "leaving"),
    ("keller_cone_flipped",            # Section 2.2.4: fan on the incoming side of the Keller cone
     "V3 d = cb * w + sb * r;", "V3 d = -cb * w + sb * r;", "leaving"),
    ("grid_without_pad",               # grid origin without its one-voxel pad
     "    org[a] = (std::floor(lo[a] / s->h) - 1.0) * s->h;", "    org[a] = (std::floor(lo[a] / s->h) - 0.0) * s->h;",
     "voxel_membership"),
    ("reception_point_first_point",    # Section 2.1: reception point = a point, not the centroid
     "      ie.rp = (1.0 / (double)(j - i)) * sum;  // reception point: centroid",
     "      ie.rp = s->pts[i];  // reception point: centroid", "rho_iterations"),
    ("edge_reception_point_at_start",  # an edge entity received at its piece's start, not middle
     "      ie.rp = E.p0 + tm * (E.p1 - E.p0);", "      ie.rp = E.p0;", "leaving"),
    ("diffraction_planes_swapped",     # Section 2.2.4: the fan ray's sector outside its planes
     "if (c.kind == CONE_DIFFRACT) return dot(r, c.tlo) >= 0.0 && dot(r, c.thi) < 0.0 && dot(r, c.rmid) > 0.0;",
     "if (c.kind == CONE_DIFFRACT) return dot(r, c.tlo) < 0.0 && dot(r, c.thi) >= 0.0 && dot(r, c.rmid) > 0.0;",
     "leaving"),
    ("binning_by_voxel",               # Section 2.1: points binned by voxel, not subvoxel
     "float t = diff / s.hs32;", "float t = diff / (2.0f * s.hs32);", "voxel_membership"),
    ("march_field_six_neighbours",     # Section 2.2.4: L1 instead of L-infinity distance
     "if (!in_grid(*s, vx + dx, vy + dy, vz + dz)) continue;",
     "if (!in_grid(*s, vx + dx, vy + dy, vz + dz) || abs(dx) + abs(dy) + abs(dz) > 1) continue;",
     "chessboard"),
    ("cone_sphere_margin_sign",        # Section 2.2.4: sphere margin subtracted from the cone
     "return t + r * sin_a >= cos_a * std::sqrt(d2 - r * r);",
     "return t - r * sin_a >= cos_a * std::sqrt(d2 - r * r);", "cone_sphere"),
    ("fibonacci_offset",               # launch lattice shifted off the zone centres
     "double z = 1.0 - (2.0 * (double)i + 1.0) / (double)N;",
     "double z = 1.0 - (2.0 * (double)i) / (double)N;", "fibonacci"),
    ("onb_v_sign",                     # basis (u, v) of the refinement, one sign flipped
     "*v = mk(b, sign + n.y * n.y * a, -n.y);", "*v = mk(b, sign + n.y * n.y * a, n.y);", "orthonormal_basis"),
    ("self_hit_any_label",             # a reflection node ignores every surface near it
     "if (e.mode == IGN_LABEL) return lbl == e.label;", "if (e.mode == IGN_LABEL) return true;", "self_hit"),
    ("self_hit_radius_doubled",        # ignore radius 2 h_s sqrt 3
     "if (dist >= r) return false;", "if (dist >= 2.0 * r) return false;", "self_hit"),
    ("reflected_axis_sign",            # Section 2.2.4: reflected cone not mirrored
     "c.axis = unit(e - 2.0 * dot(e, n) * n);", "c.axis = unit(e + 2.0 * dot(e, n) * n);", TINY),
    ("normal_orientation_dropped",     # separation plane on the far side of a surface
     "if (dot(n, e) > 0) n = -1.0 * n;", "", "facing_away"),
    ("keller_fan_exterior_and",        # Keller fan kept only where both faces see it
     "if (!(dot(d, E.n0) > 0.0 || dot(d, E.n1) > 0.0)) continue;",
     "if (!(dot(d, E.n0) > 0.0 && dot(d, E.n1) > 0.0)) continue;", "keller_point"),
    ("gradient_sign",                  # Eq. 2: e_in - e_out instead of e_in + e_out
     "V3 e = unit(I[k] - I[k - 1]) + unit(I[k] - I[k + 1]);",
     "V3 e = unit(I[k] - I[k - 1]) - unit(I[k] - I[k + 1]);", "keller_point"),
    ("reprojection_target_v_sign",     # Section 2.3: R_k = c_k + r u_k - s v_k
     "V3 R = c[k] + r * u[k] + sv * v[k];", "V3 R = c[k] + r * u[k] - sv * v[k];", TINY),
    ("edge_parameter_sign",            # Section 2.3: D_k = c_k - t w_k
     "In[k] = c[k] + tpar[k] * w[k];", "In[k] = c[k] - tpar[k] * w[k];", "keller_point"),
    ("length_last_segment_dropped",    # path length without its last segment
     "for (int k = 0; k <= n; ++k) L += norm(I[k + 1] - I[k]);",
     "for (int k = 0; k < n; ++k) L += norm(I[k + 1] - I[k]);", "los_length"),
    ("delay_scaled",                   # delay off length / c by one part in 1e9
     "ex.delay = L / C_LIGHT;", "ex.delay = L / (C_LIGHT * (1.0 + 1e-9));", TINY),
    ("kappa_farthest_first",           # Section 2.2.3: kappa keeps the farthest cone axes
     "if (a.miss != b.miss) return a.miss < b.miss;", "if (a.miss != b.miss) return a.miss > b.miss;", "kappa"),
    ("separation_plane_behind",        # Section 2.2.4: children behind the surface
     "if (c.kind == CONE_REFLECT) return dot(r, c.pn) > s.p.sep_eps;",
     "if (c.kind == CONE_REFLECT) return dot(r, c.pn) < -s.p.sep_eps;", TINY),
    ("separation_margin_dropped",      # children on the apex's own tangent plane accepted
     "if (c.kind == CONE_REFLECT) return dot(r, c.pn) > s.p.sep_eps;",
     "if (c.kind == CONE_REFLECT) return dot(r, c.pn) > -s.p.sep_eps;", TINY),
    ("child_direction_from_tx",        # incoming direction of a child taken from the TX
     "          ch.in_dir = unit(ie.rp - nd.apex);", "          ch.in_dir = unit(ie.rp - store[0].apex);", TINY),
    ("reflection_limit_plus_one",      # one reflection more than allowed
     "if (ch.nr > p.max_refl || ch.nd > p.max_diff) continue;",
     "if (ch.nr > p.max_refl + 1 || ch.nd > p.max_diff) continue;", "reflection_limit"),
    ("los_keeps_largest_miss",         # LOS miss from the farthest launch axis
     "if (it == los.end() || h.second < it->second) los[h.first] = h.second;",
     "if (it == los.end() || h.second > it->second) los[h.first] = h.second;", "los_miss"),
    ("off_edge_check_dropped",         # Section 2.3: diffraction points beyond the edge kept
     "        if (along < 0.0 || along > elen[k]) {", "        if (false) {", "leaving"),
    ("delta_validity_dropped",         # Section 2.3: paths kept whatever their gradient
     "  if (!(gn < p.delta)) { ex.status = ST_NOT_CONVERGED; return ex; }", "", "rho_iterations"),
    ("label_dedup_keeps_longest",      # Section 2.3: the longest path per label sequence
     "    if (a.length != b.length) return a.length < b.length;\n    return ie_less(a, b);",
     "    if (a.length != b.length) return a.length > b.length;\n    return ie_less(a, b);", "label_dedup"),
    ("fresnel_any_chain",              # Section 2.3: Fresnel zones across interaction chains
     "      if (!same_chain) continue;", "", "fresnel_zone_radius"),
    ("paper_launch_skips_edges",       # Section 2.2.2: the launch toward every IE misses the edges
     "        const IE& ie = s.ies[id];\n        if (ie.kind == IE_EDGE && !test_edges) continue;",
     "        const IE& ie = s.ies[id];\n        if (ie.kind == IE_EDGE) continue;", "keller_point"),
    ("kappa_plus_one",                 # Section 2.2.3: kappa + 1 coarse paths kept
     "for (size_t q = g; q < h && (int)(q - g) < p.kappa; ++q)",
     "for (size_t q = g; q < h && (int)(q - g) <= p.kappa; ++q)", "kappa"),
    ("fresnel_longest_first",          # Section 2.3: Fresnel pass in decreasing delay
     "    if (qa != qb) return qa < qb;", "    if (qa != qb) return qa > qb;", "fresnel_zone_radius"),
    ("fresnel_bins_coarse",            # delay ties in 10 cm bins instead of 1 um
     "long long qa = (long long)std::floor(a.length * 1e6), qb = (long long)std::floor(b.length * 1e6);",
     "long long qa = (long long)std::floor(a.length * 1e1), qb = (long long)std::floor(b.length * 1e1);",
     "fresnel_zone_radius"),
    ("sdf_hit_secant_dropped",         # Section 2.2.1: hit at the march point past the sign change
     "      *t_hit = t - f * (t_next - t) / (f_next - f);", "      *t_hit = t_next;", "secant_after"),
    ("reprojection_secant_sign",       # Section 2.3: secant through the wrong pair of values
     "      th = t - f * (t_next - t) / (f_next - f);", "      th = t - f * (t_next - t) / (f_next + f);",
     "middle_plane"),
    ("reprojection_probe_step_dropped",  # re-projection reading: hit at the target, no Newton step
     "      double tR_hit = std::fabs(dn) > 1e-3 ? tR - fR / dn : tR;", "      double tR_hit = tR;", "on_the_surface"),
    ("reprojection_probe_step_sign",   # re-projection reading: the Newton step from the target reversed
     "      double tR_hit = std::fabs(dn) > 1e-3 ? tR - fR / dn : tR;",
     "      double tR_hit = std::fabs(dn) > 1e-3 ? tR + fR / dn : tR;", "on_the_surface"),
    ("reprojection_probe_skipped",     # re-projection reading: the segment always marched from its end
     "    if (sdf_label(s, label, R, &fR, &nR) && std::fabs(fR) < s.p.sdf_eps) {", "    if (false) {",
     "on_the_surface"),
    ("final_visibility_dropped",       # Section 2.3: refined segments not validated by RT
     "    if (!visible(s, I[k], I[k + 1], ea, eb)) { ex.status = ST_OCCLUDED; return ex; }", "",
     "past_the_panel"),
    ("rx_sphere_at_subvoxel_centre",   # RX reception sphere centred on its subvoxel
     "    ctx.rx_sc.push_back(r);",
     "    ctx.rx_sc.push_back(mk(s.origin.x + (gs[0] + 0.5) * s.hs, s.origin.y + (gs[1] + 0.5) * s.hs,\n"
     "                           s.origin.z + (gs[2] + 0.5) * s.hs));", "rx_sphere"),
    ("fresnel_radius_misplaced_root",  # Section 2.3: sqrt(lambda a b) / (a + b)
     "double r = std::sqrt(lambda * ak * bk / (ak + bk));", "double r = std::sqrt(lambda * ak * bk) / (ak + bk);",
     "fresnel_zone_radius"),
]


def _run_mutant(tmp, name, text, planted, pins):
    src = open(SRC).read()
    if src.count(text) != 1:
        return name, None, f"the oracle holds {src.count(text)} copies of the planted text"
    cpp = os.path.join(tmp, name + ".cpp")
    with open(cpp, "w") as fh:
        fh.write(src.replace(text, planted))
    so = oracle.build_from(cpp, os.path.join(tmp, name + ".so"))
    env = dict(os.environ, NIMBUS_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"), "-q",
                        "-p", "no:cacheprovider", "-rf", "-m", "not gpu", "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_run_mutant, tmp, *m) for m in MUTANTS]
        return {name: (rc, log) for name, rc, log in (f.result() for f in futs)}


def test_unmutated_source_passes_the_same_pins():
    """The selections run clean on the oracle as it is (pytest exit 0)."""
    ks = " or ".join(f"({m[3]})" for m in MUTANTS)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"), "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu", "-k", ks],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    rc, log = outcomes[name]
    assert rc is not None, log
    # 1: some selected pin failed; 0 would mean the mistake went unnoticed, and
    # anything else (a crash, no test selected) is not a pin catching it
    assert rc == 1, f"{name}: pytest exit {rc}\n{log}"
    assert re.search(r"FAILED ", log), log


# ---------------------------------------------------------------- labelling oracle
SEG_SRC = os.path.join(ROOT, "oracle", "segment.py")

# (name, text in oracle/segment.py, planted mistake, pins expected to catch it (pytest -k))
SEGMENT_MUTANTS = [
    ("largest_eigenvector",            # group normal from the largest, not smallest, eigenvalue
     "    w, V = np.linalg.eigh(C)                      # ascending eigenvalues\n    n = V[:, 0].copy()",
     "    w, V = np.linalg.eigh(C)                      # ascending eigenvalues\n    n = V[:, 2].copy()", "box_room"),
    ("covariance_uncentred",           # covariance about the origin
     "    d = p - c\n    C = d.T @ d / m", "    d = p\n    C = d.T @ d / m", "box_room"),
    ("group_normal_unoriented",        # group normal not turned toward the input normals
     "    n = V[:, 0].copy()\n    if n @ nr.sum(axis=0) < 0.0:\n        n = -n\n    tr", "    n = V[:, 0].copy()\n    tr",
     "box_room"),
    ("spread_test_dropped",            # a single row of points counted as a plane
     "w[0] <= sp.flat_max * tr and w[1] >= sp.spread_min * tr", "w[0] <= sp.flat_max * tr", "convex_corner"),
    ("binning_by_voxel",               # groups per voxel instead of per subvoxel
     "t = (x32 - o32[None, :]) / hs32", "t = (x32 - o32[None, :]) / (2 * hs32)", "convex_corner"),
    ("join_any_angle",                 # planar neighbours joined at any angle
     "return (nor[a] @ nor[b] >= cos_join and", "return (nor[a] @ nor[b] >= -1.0 and", "folded_sheet"),
    ("join_distance_dropped",          # planar neighbours joined at any offset
     "abs(nor[a] @ (cen[b] - cen[a])) <= sp.join_dist\n                and abs(nor[b] @ (cen[a] - cen[b])) <= sp.join_dist)",
     "True)", "offset_sheets"),
    ("root_highest",                   # surfaces numbered by their last group
     "parent[max(ra, rb)] = min(ra, rb)", "parent[min(ra, rb)] = max(ra, rb)", "numbered"),
    ("relabel_dropped",                # points keep their own group's surface
     "labels[i] = surf[best] if best >= 0 else surf[g]", "labels[i] = surf[g]", "box_room"),
    ("concave_edges",                  # edges where the surfaces face each other
     "nA @ (cB - cA) < 0.0 and nB @ (cA - cB) < 0.0", "nA @ (cB - cA) > 0.0 and nB @ (cA - cB) > 0.0", "box_room"),
    ("edge_angle_reversed",            # edges only between nearly parallel surfaces
     "if not (nA @ nB <= cos_edge and", "if not (nA @ nB >= cos_edge and", "convex_corner"),
    ("edge_min_groups_ignored",        # edges between surfaces of a subvoxel or two
     "if len(members[A]) < sp.edge_min_groups or len(members[B]) < sp.edge_min_groups:", "if False:",
     "small_boxes"),
    ("edge_span_halved",               # edge ends pulled halfway in
     "edges.append(np.concatenate([x0 + min(t) * w, x0 + max(t) * w, nA, nB]))",
     "edges.append(np.concatenate([x0 + 0.5 * min(t) * w, x0 + 0.5 * max(t) * w, nA, nB]))", "convex_corner"),
    ("line_point_sign",                # point on the planes' line solved with one sign flipped
     "r = np.array([nA @ cA - nA @ mid, nB @ cB - nB @ mid])", "r = np.array([nA @ cA - nA @ mid, nB @ mid - nB @ cB])",
     "convex_corner"),
]


def _run_segment_mutant(tmp, name, text, planted, pins):
    src = open(SEG_SRC).read()
    if src.count(text) != 1:
        return name, None, f"oracle/segment.py holds {src.count(text)} copies of the planted text"
    d = os.path.join(tmp, name)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(d, "paper_2402_13747_b300"))
    for f in ("__init__.py", "config.py", "scenes.py"):
        shutil.copy(os.path.join(ROOT, "paper_2402_13747_b300", f), os.path.join(d, "paper_2402_13747_b300", f))
    os.makedirs(os.path.join(d, "tests"))
    for f in ("conftest.py", "test_segment_oracle.py", "segclouds.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests", f))
    with open(os.path.join(d, "oracle", "segment.py"), "w") as fh:
        fh.write(src.replace(text, planted))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_segment_oracle.py"), "-q",
                        "-p", "no:cacheprovider", "-rf", "-k", pins],
                       cwd=d, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def segment_outcomes(tmp_path_factory):
    oracle.build()                        # the copies carry the built C++ oracle (grid of the cloud)
    tmp = str(tmp_path_factory.mktemp("segment_mutants"))
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_run_segment_mutant, tmp, *m) for m in SEGMENT_MUTANTS]
        return {name: (rc, log) for name, rc, log in (f.result() for f in futs)}


def test_unmutated_labelling_passes_the_same_pins():
    ks = " or ".join(f"({m[3]})" for m in SEGMENT_MUTANTS)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", "test_segment_oracle.py"), "-q",
                        "-p", "no:cacheprovider", "-k", ks], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in SEGMENT_MUTANTS])
def test_labelling_pins_catch_planted_mistake(segment_outcomes, name):
    rc, log = segment_outcomes[name]
    assert rc is not None, log
    assert rc == 1, f"{name}: pytest exit {rc}\n{log}"
    assert re.search(r"FAILED ", log), log
