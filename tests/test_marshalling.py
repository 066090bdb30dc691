"""The binding's argument marshalling for lbib_add_membranes (lbib._Records),
on the CPU: every descriptor holds its body's kind, motion, vertex count and
parameters, its vertex pointers reach exactly the body's vertices (and
stress-free vertices), and its adhesion pointer reaches a record with the
body's ligand model (0 where the body has none).  Decoded through raw memory,
the way the library reads them."""
import ctypes

import numpy as np

from paper_2210_06043_gb300 import lbib
from paper_2210_06043_gb300 import workloads as wl


def _doubles(addr, n):
    return np.ctypeslib.as_array((ctypes.c_double * n).from_address(int(addr))).copy()


def _items():
    items = [(k, b) for k, c in enumerate(wl.sweep_capillaries()) for b in c.bodies]
    # a body with its own stress-free shape, and one without adhesion among them
    b0 = items[0][1]
    ref = wl.Body(b0.kind, b0.motion, b0.xy + 0.25, b0.ca, b0.beta, xy_ref=b0.xy)
    return items[:5] + [(7, ref)] + items[5:]


def test_descriptors_reach_each_bodys_data():
    items = _items()
    r = lbib._Records(items)
    assert r.descs.dtype == lbib._MEMBRANE_DT and len(r.descs) == len(items)
    assert np.array_equal(r.inst, [i for i, _ in items])
    seen_ref = seen_plain = 0
    for k, (i, b) in enumerate(items):
        d = r.descs[k]
        nv = len(b.xy)
        assert (int(d["kind"]), int(d["motion"]), int(d["nv"])) == (int(b.kind), int(b.motion), nv)
        assert (float(d["ca"]), float(d["beta"]), float(d["ka"]), float(d["density_ratio"])) == \
            (float(b.ca), float(b.beta), float(b.ka), float(b.density_ratio))
        assert np.array_equal(_doubles(d["xy"], 2 * nv), np.asarray(b.xy, np.float64).ravel())
        if b.xy_ref is None:
            assert int(d["xy_ref"]) == 0
            seen_plain += 1
        else:
            assert np.array_equal(_doubles(d["xy_ref"], 2 * nv), np.asarray(b.xy_ref, np.float64).ravel())
            seen_ref += 1
        a = b.adhesion
        if a is None:
            assert int(r.adh_ptr[k]) == 0
        else:
            raw = (ctypes.c_char * lbib._ADHESION_DT.itemsize).from_address(int(r.adh_ptr[k]))
            rec = np.frombuffer(bytes(raw), lbib._ADHESION_DT)[0]
            assert int(rec["n_ligands"]) == int(a.n_lig)
            assert [float(rec[f]) for f in ("sigma", "y_cr", "y_eq", "kf_dt", "kr0_dt", "xi")] == \
                [float(a.sigma), float(a.y_cr), float(a.y_eq), float(a.kf_dt), float(a.kr0_dt), float(a.xi)]
    assert seen_ref == 1 and seen_plain == len(items) - 1
    assert sorted(r.with_adh) == [k for k, (_, b) in enumerate(items) if b.adhesion is not None]


def test_empty_and_single_body():
    r = lbib._Records([])
    assert len(r.descs) == 0 and len(r.adh_ptr) == 0
    b = wl.sweep_capillaries()[0].bodies[0]
    r = lbib._Records([(3, b)])
    assert int(r.descs[0]["nv"]) == len(b.xy) and int(r.inst[0]) == 3
