"""Power-iteration checkpoint and resume: a run stopped after some batches,
saved to a file and resumed in a fresh problem, continues with the same
histories and eigenvalues as an uninterrupted run (k per batch, the last
batch's event log and the tallies bit-equal); mismatched, damaged or foreign
states are refused."""
import numpy as np
import pytest

from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_logs_equal

pytestmark = pytest.mark.gpu

NPB, NI, NA = 20_000, 2, 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_00263_gb300 import build
    build.build()


def _opts(scheme=tb.SCHEME_ASYNC, seed=4):
    return tb.RunOpts(seed=seed, scheme=scheme, decomposition=tb.DECOMP_MONO, want_event_log=True)


def _finish(prob, r):
    return {"k": r["k_batch"], "kmean": r["k_mean"], "log": prob.event_log(int(r["n_source"][-1])),
            "mesh": prob.tally(tb.TALLY_MESH), "scal": prob.tally(tb.TALLY_SCALARS),
            "mesh_sd": prob.tally(tb.TALLY_MESH, stddev=True), "final": r["final_by_type"], "done": r["batches_done"]}


def _check_same(a, b):
    assert np.array_equal(a["k"], b["k"]), (a["k"], b["k"])
    assert a["kmean"] == b["kmean"] and a["done"] == b["done"] == NI + NA
    assert_logs_equal(a["log"], b["log"], "last batch")
    assert np.array_equal(a["final"], b["final"])
    # tallies are order-independent fixed-point sums: a resumed run gives the
    # uninterrupted run's bits
    for key in ("mesh", "scal", "mesh_sd"):
        assert np.array_equal(a[key].view(np.uint64), b[key].view(np.uint64)), key


@pytest.mark.parametrize("scheme", [tb.SCHEME_ASYNC, tb.SCHEME_STACK], ids=["async", "stack"])
def test_resume_from_file_equals_uninterrupted_run(scheme, tmp_path):
    spec = inputs.c5g7_lattice()
    full = tb.Problem(spec)
    ref = _finish(full, full.power_iteration(NPB, NI, NA, _opts(scheme)))
    full.close()

    p1 = tb.Problem(spec)
    part = p1.power_iteration(NPB, NI, NA, _opts(scheme), stop_after=3)
    assert part["batches_done"] == 3
    with pytest.raises(tb.TransportError):
        p1.tally(tb.TALLY_MESH)          # tallies are final only at the end
    path = tmp_path / "eig.ckpt"
    path.write_bytes(p1.eig_checkpoint())
    p1.close()

    p2 = tb.Problem(spec)
    r = p2.power_iteration(NPB, NI, NA, _opts(scheme), resume=path.read_bytes())
    got = _finish(p2, r)
    assert np.array_equal(got["k"][:3], part["k_batch"][:3])
    _check_same(ref, got)
    p2.close()


def test_chained_stops_and_refusals():
    spec = inputs.c5g7_lattice()
    full = tb.Problem(spec)
    ref = _finish(full, full.power_iteration(NPB, NI, NA, _opts()))
    with pytest.raises(tb.TransportError) as e:
        full.eig_checkpoint()                    # ran to the end: nothing kept
    assert e.value.status == tb.TR_ERR_STATE
    full.close()

    p = tb.Problem(spec)
    p.power_iteration(NPB, NI, NA, _opts(), stop_after=2)
    s2 = p.eig_checkpoint()
    r = p.power_iteration(NPB, NI, NA, _opts(), stop_after=5, resume=s2)
    assert r["batches_done"] == 5
    s5 = p.eig_checkpoint()
    got = _finish(p, p.power_iteration(NPB, NI, NA, _opts(), resume=s5))
    _check_same(ref, got)

    for bad_opts, bad_state, status in ((_opts(seed=5), s2, tb.TR_ERR_STATE),
                                        (_opts(), b"XXXXXXXX" + s2[8:], tb.TR_ERR_INVALID),
                                        (_opts(), s2[:-8], tb.TR_ERR_INVALID)):
        with pytest.raises(tb.TransportError) as e:
            p.power_iteration(NPB, NI, NA, bad_opts, resume=bad_state)
        assert e.value.status == status
    p.close()


def _bank_view(state):
    """(N, offset of the source bank) of a serialised state: the bank (x, y,
    z doubles, group int32, packed cell uint32, N each) ends the buffer; N is
    the header's third 64-bit word."""
    n = int(np.frombuffer(state, np.uint64, 1, 24)[0])
    return n, len(state) - 32 * n


def test_tampered_or_foreign_checkpoints_are_refused():
    """Every restored source site is checked on the host before anything is
    uploaded (group in range, cell inside the grid, pin bit only where a pin
    is, position finite and inside its cell), and the state carries a
    fingerprint of the problem it came from."""
    spec = inputs.c5g7_lattice()
    nz, ny, nx = spec.shape
    p = tb.Problem(spec)
    p.power_iteration(NPB, NI, NA, _opts(), stop_after=2)
    s = bytes(p.eig_checkpoint())
    n, off = _bank_view(s)
    assert n > 0 and off > 0
    X, Y, Z, G, CELL = 0, 8 * n, 16 * n, 24 * n, 28 * n
    dt = {X: np.float64, Y: np.float64, Z: np.float64, G: np.int32, CELL: np.uint32}

    def patched(i, **fields):
        b = bytearray(s)
        for name, value in fields.items():
            f = {"x": X, "y": Y, "z": Z, "g": G, "cell": CELL}[name]
            a = np.frombuffer(b, dt[f], n, off + f)
            a.setflags(write=True)
            a[i] = value
        return bytes(b)

    cells = np.frombuffer(s, np.uint32, n, off + CELL)
    k0 = (int(cells[0]) >> 20) & 1023
    # site 0 moved into the radial reflector cell (no pin), position inside it
    refl = (nx - 1) | ((ny - 1) << 10) | (k0 << 20)
    xr, yr = 0.5 * (spec.x_planes[-2] + spec.x_planes[-1]), 0.5 * (spec.y_planes[-2] + spec.y_planes[-1])
    bad_states = [
        patched(0, g=7),                                       # group G
        patched(n - 1, g=-1),                                  # negative group
        patched(3, cell=int(cells[3]) | 1023),                 # cell index beyond the grid
        patched(5, cell=int(cells[5]) | (1 << 31)),            # stray high bit
        patched(1, x=np.nan),                                  # non-finite position
        patched(2, y=1e6),                                     # position outside its cell
        patched(0, x=xr, y=yr, cell=refl | (1 << 30)),         # pin bit where the cell has no pin
    ]
    for bad in bad_states:
        with pytest.raises(tb.TransportError) as e:
            p.power_iteration(NPB, NI, NA, _opts(), resume=bad)
        assert e.value.status == tb.TR_ERR_INVALID
    # the same move without the pin bit is a valid site: the run resumes
    r = p.power_iteration(NPB, NI, NA, _opts(), resume=patched(0, x=xr, y=yr, cell=refl))
    assert r["batches_done"] == NI + NA
    # the same shapes but other cross sections: a foreign state
    q = tb.Problem(inputs.c5g7_lattice(xs_seed=2026))
    with pytest.raises(tb.TransportError) as e:
        q.power_iteration(NPB, NI, NA, _opts(), resume=s)
    assert e.value.status == tb.TR_ERR_STATE
    q.close()
    # the untouched state still resumes
    r = p.power_iteration(NPB, NI, NA, _opts(), resume=s)
    assert r["batches_done"] == NI + NA
    p.close()
