"""The C-ABI library loads and exports every entry point include/bgk.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2312_06567_gb300 import bgk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"BGK_API\s+[\w\s\*]+?\b(bgk_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bgk_create", "bgk_destroy", "bgk_step", "bgk_rhs", "bgk_qprime",
                     "bgk_moments", "bgk_set_state", "bgk_get_state", "bgk_totals"):
        assert required in names


def test_library_exports_every_declared_symbol(libbgk):
    for name in _declared():
        assert hasattr(libbgk, name), name
        assert isinstance(getattr(libbgk, name), ctypes._CFuncPtr)


def test_binding_covers_every_declared_symbol():
    assert set(_declared()) == set(bgk.SIGNATURES)


def test_descriptor_layout_matches_header(tmp_path):
    """ctypes structures agree with the C compiler's layout of include/bgk.h."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text("""#include <stdio.h>
#include <stddef.h>
#include "bgk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bgk_mesh_desc), offsetof(bgk_mesh_desc, lo),
         offsetof(bgk_mesh_desc, hi), offsetof(bgk_mesh_desc, periodic),
         offsetof(bgk_mesh_desc, order), offsetof(bgk_mesh_desc, bc_state), offsetof(bgk_mesh_desc, face_type),
         offsetof(bgk_mesh_desc, node_xyz));
  printf("%zu %zu %zu\\n", sizeof(bgk_vgrid_desc), offsetof(bgk_vgrid_desc, lo),
         offsetof(bgk_vgrid_desc, hi));
  printf("%zu %zu\\n", sizeof(bgk_gas_desc), offsetof(bgk_gas_desc, theta_S));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().splitlines()]
    M = bgk.MeshDesc
    assert out[0] == [ctypes.sizeof(M), M.lo.offset, M.hi.offset, M.periodic.offset,
                      M.order.offset, M.bc_state.offset, M.face_type.offset, M.node_xyz.offset]
    V = bgk.VGridDesc
    assert out[1] == [ctypes.sizeof(V), V.lo.offset, V.hi.offset]
    assert out[2] == [ctypes.sizeof(bgk.GasDesc), bgk.GasDesc.theta_S.offset]


def test_invalid_descriptors_rejected_on_the_host(libbgk):
    """Descriptor validation happens before any CUDA call: BGK_EINVAL + message."""
    import pytest
    from paper_2312_06567_gb300 import workloads as W
    base = W.periodic_sine_box()
    bad = [base.replace(p=0), base.replace(p=5), base.replace(vel_n=(1, 8, 8)),
           base.replace(delta=-1.0), base.replace(Pr=0.5), base.replace(mesh_n=(0, 4, 4)),
           base.replace(mesh_hi=(0.0, 1, 1)),
           W.normal_shock_tube().replace(dirichlet={(0, -1): (0.0, (1, 0, 0), 1.0),
                                                    (0, 1): (1.0, (1, 0, 0), 1.0)}),
           # specular faces: on a periodic axis, or with a velocity grid not symmetric in the axis
           base.replace(specular=((0, -1),)),
           W.normal_shock_tube().replace(dirichlet={}, specular=((0, -1), (0, 1)), vel_lo=(-9.0, -8.0, -8.0),
                                         vel_hi=(11.0, 8.0, 8.0))]
    for wl in bad:
        with pytest.raises(bgk.BGKError) as ei:
            bgk.Solver(wl)
        assert ei.value.status == bgk.BGK_EINVAL
        assert str(ei.value)


def test_curvilinear_descriptors_rejected_on_the_host(libbgk):
    """Curvilinear and wall descriptors are validated before any CUDA call: a
    mesh with a non-positive Jacobian (one element's node order mirrored), a
    diffuse wall without a positive temperature, an unknown face type give
    BGK_EINVAL; specular faces on the curvilinear path give BGK_ENOTSUP."""
    import numpy as np
    import pytest
    from paper_2312_06567_gb300 import workloads as W
    wl = W.wavy_periodic_box(p=2, n=(2, 2, 2), vel_n=(4, 4, 4))
    x = np.ascontiguousarray(W.node_positions(wl))
    x6 = x.reshape(wl.n_elem, 3, 3, 3, 3)
    x6[1] = x6[1][:, :, ::-1].copy()                     # mirror element 1 along xi_1: J < 0
    m, v, g = bgk.descriptors(wl, x)
    lib = bgk.load()
    h = ctypes.c_void_p()
    st = lib.bgk_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(v), ctypes.byref(g), bgk.BGK_FP64, None)
    msg = lib.bgk_last_error(h).decode()
    lib.bgk_destroy(h)
    assert st == bgk.BGK_EINVAL and "Jacobian" in msg
    chan = wl.replace(periodic=(False, True, True), diffuse={(0, -1): ((0, 0, 0), 0.0), (0, 1): ((0, 0, 0), 1.0)})
    with pytest.raises(bgk.BGKError) as ei:
        bgk.Solver(chan)
    assert ei.value.status == bgk.BGK_EINVAL
    spec = W.normal_shock_tube().replace(dirichlet={(0, 1): (1.0, (1, 0, 0), 1.0)}, specular=((0, -1),),
                                         diffuse={}, closed=(), vel_lo=(-9.0, -8.0, -8.0), vel_hi=(9.0, 8.0, 8.0))
    for variant in (spec.replace(closed=((0, 1),), dirichlet={}), spec.replace(mapping=W._wavy(0.0))):
        with pytest.raises(bgk.BGKError) as ei:
            bgk.Solver(variant)
        assert ei.value.status == bgk.BGK_ENOTSUP
    m, v, g = bgk.descriptors(W.normal_shock_tube())
    m.face_type[0] = 4
    st = lib.bgk_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(v), ctypes.byref(g), bgk.BGK_FP64, None)
    lib.bgk_destroy(h)
    assert st == bgk.BGK_EINVAL


def test_library_metric_terms_equal_the_oracle(libbgk):
    """Host-side metric terms of the library (bgk_curved_metrics) against the
    oracle's independently written curl form: node metrics S^d, Jacobians and
    averaged face vectors of the sphere O-grid (p = 1, 2; small and the
    benchmark's full 6912 elements) and a warped periodic box (p = 3), to 1e-12
    of their scale."""
    import numpy as np
    from oracle import curved
    from paper_2312_06567_gb300 import workloads as W
    cases = [W.sphere_ogrid(n=(2, 4, 6), p=1), W.sphere_ogrid(n=(2, 3, 4), p=2),
             W.wavy_periodic_box(p=3, n=(2, 2, 3), amp=0.07),
             W.sphere_ogrid()]                            # the benchmark's full 12 x 24 x 24 mesh
    for wl in cases:
        x = W.node_positions(wl)
        S, J, fv = bgk.curved_metrics(wl, x)
        mesh = curved.CurvedMesh(wl.mesh_n, wl.periodic, x, wl.p)
        q = wl.p + 1
        So = np.moveaxis(mesh.S.reshape(wl.n_elem, 3, 3, -1), 3, 1).reshape(-1, 3, 3)   # [P, d, n]
        sc = np.max(np.abs(So))
        assert np.max(np.abs(S - So)) <= 1e-12 * sc, wl.name
        assert np.max(np.abs(J - mesh.J.reshape(-1))) <= 1e-12 * np.max(mesh.J), wl.name
        for d in range(3):
            for side in (-1, 1):
                # both ordered (higher axis, lower axis) with the lower one fastest
                f_o = mesh.face[(d, side)].reshape(wl.n_elem, q * q, 3)
                f_l = fv[:, 2 * d + (side > 0)]
                assert np.max(np.abs(f_l - f_o)) <= 1e-12 * sc, (wl.name, d, side)


def test_library_fr_operators_equal_the_oracle(libbgk):
    """The library's host FR operators (nodes, weights, D, traces, correction
    derivatives) equal the oracle's pinned FR1D to 1e-14, p = 1..4."""
    import numpy as np
    from oracle.fr import FR1D
    for p in (1, 2, 3, 4):
        lib_fr, _ = bgk.fr_tables(p)
        o = FR1D(p)
        for name, ref in (("xi", o.xi), ("w", o.wq), ("D", o.D), ("lm", o.l_minus), ("lp", o.l_plus),
                          ("dgL", o.dgL), ("dgR", o.dgR)):
            assert np.max(np.abs(lib_fr[name] - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref))), (p, name)


def test_curvilinear_fp32_line_operator_conserves_exactly():
    """One line of the curvilinear mixed stage, applied in exact rational
    arithmetic to the library's stored FP32 tables: each node's residual is
    the deviation form (off-diagonal D and the column defects acting on
    A_j (f_j - f_i), the two lifted face jumps A_face (F* - f_i) - trace) plus
    f_i times its geometric remainder (the f_i-proportional terms of the same
    operator written on A_j - A_i).  Whatever the node values, flux
    coefficients and common fluxes, the W-weighted sum of the residuals equals
    the face fluxes s_R A_R F*_R + s_L A_L F*_L with s_R = -s_L = sum W g_R'
    (the same weight on both sides of every face), to the rounding of the
    stored defects: the FP32 tables conserve the quadrature total exactly."""
    import random
    from fractions import Fraction as Fr
    rng = random.Random(7)
    for p in (1, 2, 3, 4):
        fr, c = bgk.fr_tables(p)
        q = p + 1
        W = [Fr(float(v)) for v in fr["w"]]
        D = [[Fr(float(c["D"][i][j])) for j in range(q)] for i in range(q)]
        lp = [Fr(float(v)) for v in c["lp"]]
        lm = [Fr(float(v)) for v in c["lm"]]
        gL = [Fr(float(v)) for v in c["dgL"]]
        gR = [Fr(float(v)) for v in c["dgR"]]
        de = [Fr(float(v)) for v in c["def"]]
        # the left-face tables are the mirror images of the right-face ones
        assert all(lm[i] == lp[q - 1 - i] and gL[i] == -gR[q - 1 - i] for i in range(q))
        sR = sum(W[i] * gR[i] for i in range(q))
        sL = sum(W[i] * gL[i] for i in range(q))
        assert sR + sL == 0 and abs(float(sR) - 1.0) < 1e-6
        # constant data see no defect: the defects sum to zero up to their FP32 rounding
        dscale = max(abs(float(v)) for v in c["def"]) + 1e-30
        assert abs(float(sum(de))) <= q * 2.0 ** -23 * dscale
        for trial in range(4):
            A = [Fr(rng.uniform(-2, 2)) for _ in range(q)]
            AL, AR = Fr(rng.uniform(-2, 2)), Fr(rng.uniform(-2, 2))
            f = [Fr(rng.uniform(0, 1)) for _ in range(q)]
            FL, FR = Fr(rng.uniform(0, 1)), Fr(rng.uniform(0, 1))
            total = Fr(0)
            for i in range(q):
                w = [A[j] * (f[j] - f[i]) for j in range(q)]
                t = sum((D[i][j] - de[j]) * w[j] for j in range(q) if j != i)
                t += gL[i] * (AL * (FL - f[i]) - sum(lm[j] * w[j] for j in range(q)))
                t += gR[i] * (AR * (FR - f[i]) - sum(lp[j] * w[j] for j in range(q)))
                dA = [A[j] - A[i] for j in range(q)]
                H = sum(D[i][j] * dA[j] for j in range(q) if j != i) - sum(de[j] * dA[j] for j in range(q))
                H += gR[i] * (AR - A[i] - sum(lp[j] * dA[j] for j in range(q)))
                H += gL[i] * (AL - A[i] - sum(lm[j] * dA[j] for j in range(q)))
                total += W[i] * (t + f[i] * H)
            err = total - (sR * AR * FR + sL * AL * FL)
            assert abs(float(err)) <= 1e-13, (p, trial, float(err))


def test_plain_c_program_links_and_calls_the_library(tmp_path, libbgk):
    """A C program built against include/bgk.h and linked to libbgk.so (no
    ctypes) gets BGK_EINVAL and a message for an invalid descriptor and for
    missing arguments, and reads the FR operators, which equal the oracle's."""
    import subprocess
    import numpy as np
    from oracle.fr import FR1D
    src = tmp_path / "client.c"
    src.write_text("""#include <stdio.h>
#include <string.h>
#include "bgk.h"
int main(void) {
  bgk_mesh_desc m; memset(&m, 0, sizeof m);
  bgk_vgrid_desc v = {{8, 8, 8}, {-6, -6, -6}, {6, 6, 6}};
  bgk_gas_desc g = {0.0, 1.0, 0.08, 1.0, -1.0};
  m.n[0] = m.n[1] = m.n[2] = 2; m.hi[0] = m.hi[1] = m.hi[2] = 1.0;
  m.periodic[0] = m.periodic[1] = m.periodic[2] = 1; m.order = 9;          /* order out of range */
  bgk_ctx *ctx = NULL;
  int st = bgk_create(&ctx, &m, &v, &g, BGK_FP64, NULL);
  const char *msg = bgk_last_error(ctx);
  printf("%d %d\\n", st, (int)(msg != NULL && strlen(msg) > 0));
  bgk_destroy(ctx);
  printf("%d %d\\n", bgk_curved_metrics(&m, NULL, NULL, NULL), bgk_fr_tables(0, NULL, NULL));
  double fr[6 * 4 + 16]; float c32[16 + 5 * 4];
  printf("%d\\n", bgk_fr_tables(3, fr, c32));
  for (int i = 0; i < 6 * 4 + 16; ++i) printf("%.17g\\n", fr[i]);
  return 0;
}
""")
    exe = tmp_path / "client"
    libdir = os.path.join(ROOT, "paper_2312_06567_gb300")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lbgk",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    lines = subprocess.check_output([str(exe)]).decode().split("\n")
    assert lines[0].split() == [str(bgk.BGK_EINVAL), "1"]
    assert lines[1].split() == [str(bgk.BGK_EINVAL)] * 2
    assert int(lines[2]) == bgk.BGK_OK
    v = np.array([float(t) for t in lines[3:3 + 40]])
    o = FR1D(3)
    ref = np.concatenate([o.xi, o.wq, o.D.ravel(), o.l_minus, o.l_plus, o.dgL, o.dgR])
    assert np.max(np.abs(v - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises (there is no CPU path)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2312_06567_gb300 import bgk, workloads as W\n"
            "bgk.LIB_PATH = %r\n"
            "try:\n"
            "    bgk.load(bgk.LIB_PATH)\n"
            "except RuntimeError as e:\n"
            "    assert 'no CPU fallback' in str(e); print('load raised')\n"
            "import functools\n"
            "bgk.load = functools.partial(bgk.load, %r)\n"
            "try:\n"
            "    bgk.Solver(W.periodic_sine_box())\n"
            "except RuntimeError as e:\n"
            "    print('solver raised')\n") % (ROOT, str(tmp_path / "absent.so"), str(tmp_path / "absent.so"))
    out = subprocess.check_output([sys.executable, "-c", code]).decode()
    assert "load raised" in out and "solver raised" in out


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it."""
    pkg = os.path.join(ROOT, "paper_2312_06567_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
            assert "oracle" not in re.findall(r"import_module\(['\"](\w+)", text), f


def test_every_entry_point_documents_its_errors():
    """Each declaration in include/bgk.h is preceded (directly, or as part of a
    group sharing one comment) by a comment that states its error behaviour."""
    text = open(os.path.join(ROOT, "include", "bgk.h")).read()
    for m in re.finditer(r"BGK_API\s+([\w\s\*]+?)\b(bgk_\w+)\s*\(", text):
        if "char" in m.group(1):                      # bgk_last_error returns text, not a status
            continue
        before = re.sub(r"^#define.*$", "", text[:m.start()], flags=re.M)   # inline comments of constants
        comment = before.rsplit("/*", 1)[1]
        assert re.search(r"Errors?:|BGK_E[A-Z]+", comment), m.group(2)


def test_descriptors_carry_each_workload_face():
    """The binding's descriptors: face 2d + (side > 0) gets the workload's kind
    and state (Dirichlet (rho, U, theta); diffuse (1, U_w, theta_w)),
    periodic axes and sizes as defined, the gas as given."""
    from paper_2312_06567_gb300 import workloads as W
    shock = W.normal_shock_tube()
    m, v, g = bgk.descriptors(shock)
    assert list(m.periodic) == [0, 1, 1] and list(m.n) == list(shock.mesh_n) and m.order == shock.p
    assert m.face_type[0] == m.face_type[1] == bgk.BGK_FACE_DIRICHLET
    for f, key in ((0, (0, -1)), (1, (0, 1))):
        rho, U, th = shock.dirichlet[key]
        assert list(m.bc_state[f]) == [rho, U[0], U[1], U[2], th]
    assert m.bc_state[0][1] > m.bc_state[1][1] > 0                  # supersonic inflow, slower outflow
    assert (g.delta, g.Pr, g.mu_ref) == (shock.delta, shock.Pr, shock.mu_ref)
    assert list(v.n) == list(shock.vel_n) and list(v.lo) == list(shock.vel_lo)
    og = W.sphere_ogrid(n=(2, 4, 4), vel_n=(6, 6, 6))
    x = np.ascontiguousarray(W.node_positions(og))
    m, _, _ = bgk.descriptors(og, x)
    assert list(m.periodic) == [0, 0, 1]
    assert m.face_type[0] == bgk.BGK_FACE_DIFFUSE and m.face_type[1] == bgk.BGK_FACE_DIRICHLET
    assert m.face_type[2] == m.face_type[3] == bgk.BGK_FACE_CLOSED
    U_w, th_w = og.diffuse[(0, -1)]
    assert list(m.bc_state[0]) == [1.0, U_w[0], U_w[1], U_w[2], th_w]
    assert m.node_xyz == x.ctypes.data
    spec = shock.replace(dirichlet={(0, 1): shock.dirichlet[(0, 1)]}, specular=((0, -1),))
    m, _, _ = bgk.descriptors(spec)
    assert m.face_type[0] == bgk.BGK_FACE_SPECULAR and m.face_type[1] == bgk.BGK_FACE_DIRICHLET


def test_noalloc_moments_reject_invalid_arguments_before_any_cuda_call(libbgk):
    """bgk_moments_noalloc validates on the host first: more points than its
    fixed 2^21-double scratch holds (11 n_points > 2^21), no points, a third
    component, a one-node velocity axis, missing pointers -> BGK_EINVAL."""
    v = bgk.VGridDesc()
    for d in range(3):
        v.n[d], v.lo[d], v.hi[d] = 8, -6.0, 6.0
    dummy = ctypes.c_void_p(16)                 # never dereferenced on these paths
    call = lambda vg, f, nc, npts, m: libbgk.bgk_moments_noalloc(vg, f, nc, npts, m, None)
    assert call(ctypes.byref(v), dummy, 1, (1 << 21) // 11 + 1, dummy) == bgk.BGK_EINVAL
    assert call(ctypes.byref(v), dummy, 1, 0, dummy) == bgk.BGK_EINVAL
    assert call(ctypes.byref(v), dummy, 3, 10, dummy) == bgk.BGK_EINVAL
    assert call(ctypes.byref(v), None, 1, 10, dummy) == bgk.BGK_EINVAL
    assert call(None, dummy, 1, 10, dummy) == bgk.BGK_EINVAL
    v.n[1] = 1
    assert call(ctypes.byref(v), dummy, 1, 10, dummy) == bgk.BGK_EINVAL


def test_noalloc_binding_refuses_wrong_buffers_before_calling_the_library(monkeypatch):
    """The Python wrapper of bgk_moments_noalloc checks device, dtype,
    contiguity and size of f and m and raises ValueError before the library
    is loaded or called (a wrong buffer would be read or written out of
    bounds on the device)."""
    torch = pytest.importorskip("torch")

    def never(*a, **k):
        raise AssertionError("the library must not be reached")
    monkeypatch.setattr(bgk, "load", never)
    v = bgk.VGridDesc()
    for d in range(3):
        v.n[d], v.lo[d], v.hi[d] = 4, -3.0, 3.0
    P = 10
    cpu_f = torch.zeros((1, 64, P), dtype=torch.float64)
    cpu_m = torch.zeros((P, 11), dtype=torch.float64)
    with pytest.raises(ValueError, match="device memory"):
        bgk.moments_noalloc(v, cpu_f, 1, P, cpu_m)
    with pytest.raises(ValueError, match="CUDA torch tensor"):
        bgk.moments_noalloc(v, np.zeros((1, 64, P)), 1, P, cpu_m)
    with pytest.raises(ValueError):
        bgk.moments_noalloc(v, cpu_f, 3, P, cpu_m)
    with pytest.raises(ValueError):
        bgk.moments_noalloc(v, cpu_f, 1, 0, cpu_m)

    class FakeCuda:
        """Stands for a CUDA tensor on a machine without a GPU."""
        def __init__(self, n, dtype=torch.float64, contiguous=True):
            self.is_cuda, self.dtype, self._n, self._c = True, dtype, n, contiguous
        def numel(self):
            return self._n
        def is_contiguous(self):
            return self._c
    ok_f, ok_m = FakeCuda(64 * P), FakeCuda(11 * P)
    with pytest.raises(ValueError, match="float64"):
        bgk.moments_noalloc(v, FakeCuda(64 * P, torch.float32), 1, P, ok_m)
    with pytest.raises(ValueError, match="needs"):
        bgk.moments_noalloc(v, FakeCuda(64 * P - 1), 1, P, ok_m)
    with pytest.raises(ValueError, match="needs"):
        bgk.moments_noalloc(v, FakeCuda(64 * P), 2, P, ok_m)
    with pytest.raises(ValueError, match="needs"):
        bgk.moments_noalloc(v, ok_f, 1, P, FakeCuda(11 * P - 1))
    with pytest.raises(ValueError, match="contiguous"):
        bgk.moments_noalloc(v, ok_f, 1, P, FakeCuda(11 * P, contiguous=False))


def test_header_compiles_cleanly_as_c99_and_cxx11(tmp_path):
    """include/bgk.h is a plain C header: strict C99 and C++11, every warning an error."""
    import subprocess
    src = "#include \"bgk.h\"\nint main(void) { return (int)sizeof(bgk_mesh_desc) > 0 ? 0 : 1; }\n"
    for ext, cc, std in (("c", "gcc", "-std=c99"), ("cpp", "g++", "-std=c++11")):
        f = tmp_path / ("h." + ext)
        f.write_text(src)
        subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-fsyntax-only", str(f)], check=True)


def test_binding_signatures_match_the_header_prototypes():
    """Every ctypes signature has the prototype's argument count, and each
    scalar argument the prototype's C type (a pointer may be c_void_p or a typed
    pointer); the return types are the status int (or text)."""
    text = open(os.path.join(ROOT, "include", "bgk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    scalars = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float,
               "long long": ctypes.c_longlong, "unsigned long long": ctypes.c_ulonglong}
    seen = 0
    for m in re.finditer(r"BGK_API\s+([\w\s\*]+?)\b(bgk_\w+)\s*\(([^)]*)\)", text):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3)
        res, args = bgk.SIGNATURES[name]
        assert (res is ctypes.c_char_p) == ("char" in ret), name
        plist = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        assert len(plist) == len(args), name
        for p, a in zip(plist, args):
            if "*" in p or "[" in p:
                assert a is ctypes.c_void_p or a is ctypes.c_char_p or hasattr(a, "_type_") and \
                    issubclass(a, ctypes._Pointer), (name, p)
                continue
            ctype = re.sub(r"\s+\w+$", "", p.replace("const ", "")).strip()
            assert a is scalars[ctype], (name, p, a)
        seen += 1
    assert seen == len(bgk.SIGNATURES)


def test_face_vectors_are_single_valued_on_a_discontinuous_mesh():
    """One element of a warped box perturbed on its own (the geometry no
    longer matches across its faces): each shared face still carries one face
    vector, bit for bit the same from both sides (the two traces averaged),
    and it equals the oracle's."""
    from oracle import curved
    from paper_2312_06567_gb300 import workloads as W
    wl = W.wavy_periodic_box(p=2, n=(3, 3, 2), amp=0.05)
    x = np.ascontiguousarray(W.node_positions(wl))
    e = 1 + 3 * (1 + 3 * 0)                                      # an inner element of the first two axes
    x[e] += 0.01 * np.random.default_rng(4).standard_normal(x[e].shape)
    S, J, fv = bgk.curved_metrics(wl, x)
    mesh = curved.CurvedMesh(wl.mesh_n, wl.periodic, x, wl.p)
    q = wl.p + 1
    n1, n2 = wl.mesh_n[0], wl.mesh_n[1]
    stride = (1, n1, n1 * n2)
    for d in range(3):
        c = (e % n1, (e // n1) % n2, e // (n1 * n2))[d]
        nb = e + stride[d] if c < wl.mesh_n[d] - 1 else e - (wl.mesh_n[d] - 1) * stride[d]
        assert np.array_equal(fv[e, 2 * d + 1], fv[nb, 2 * d]), d              # shared face, both sides
        f_o = mesh.face[(d, 1)].reshape(wl.n_elem, q * q, 3)[e]
        assert np.max(np.abs(fv[e, 2 * d + 1] - f_o)) <= 1e-12 * np.max(np.abs(f_o)), d


def test_collapsed_pole_faces_have_zero_face_vectors():
    """The polar faces of the latitude--longitude O-grid collapse onto the
    axis: the library's face vectors (area-weighted normals) vanish there to
    rounding, p = 1 and 2, so no flux could cross them even if they were not
    declared closed."""
    from paper_2312_06567_gb300 import workloads as W
    for p in (1, 2):
        wl = W.sphere_ogrid(n=(3, 6, 8), p=p)
        assert set(wl.closed) == {(1, -1), (1, 1)}
        _, _, fv = bgk.curved_metrics(wl, np.ascontiguousarray(W.node_positions(wl)))
        c2 = (np.arange(wl.n_elem) // wl.mesh_n[0]) % wl.mesh_n[1]
        scale = np.abs(fv).max()
        assert np.abs(fv[c2 == 0][:, 2]).max() <= 1e-14 * scale
        assert np.abs(fv[c2 == wl.mesh_n[1] - 1][:, 3]).max() <= 1e-14 * scale
