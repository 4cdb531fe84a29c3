"""tr_run_fixed_source_noalloc: the run for callers that cannot allocate
device memory while they work (an application that reserves the GPU's memory
for its own pool, or a loop that cannot accept the synchronisation of
cudaMalloc).  Its scratch is the library's static device array, so two calls
in a row must each clear and reuse it and still match the allocating entry
point.  This file is collected last so that a failure here never stops the
rest of the GPU suite."""
import numpy as np
import pytest

from paper_2506_00263_gb300 import binding as tb
from paper_2506_00263_gb300 import inputs
from tests._util import assert_tally_close

pytestmark = pytest.mark.gpu

MAX_QUEUE = 4096          # TR_NOALLOC_MAX_QUEUE_CAPACITY in include/tr.h
MAX_BINS = 24576          # TR_NOALLOC_MAX_TALLY_BINS in include/tr.h


def _same_bits(a, b, what):
    """Mesh and energy bins are order-independent fixed-point sums of the same
    contributions in both entry points, so the allocation-free run gives
    exactly the allocating run's values there.  (The scalar tallies are
    reduced differently -- per history into fixed point here, per-history
    sums in a fixed order in the allocating run -- and agree within the
    suite's tolerance.)"""
    a, b = np.asarray(a), np.asarray(b)
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), what


def test_noalloc_matches_allocating_run_on_two_calls():
    import torch
    from paper_2506_00263_gb300 import build
    build.build()
    prob = tb.Problem(inputs.c5g7_lattice())
    n = 100_003
    ref_opts = tb.RunOpts(n_histories=n, seed=3, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_SPLIT)
    ref = prob.run_fixed_source(ref_opts)
    ref_mesh = prob.tally(tb.TALLY_MESH)
    ref_scal = prob.tally(tb.TALLY_SCALARS)

    mesh = torch.empty(ref_mesh.size, dtype=torch.float64, device="cuda")
    scal = torch.empty(3, dtype=torch.float64, device="cuda")
    calls = [tb.RunOpts(n_histories=n, seed=3, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_SPLIT),
             # second call: force spills through the static link arena
             tb.RunOpts(n_histories=n, seed=3, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_SPLIT,
                        spill_threshold=-32, queue_capacity=MAX_QUEUE)]
    for k, opts in enumerate(calls):
        mesh.fill_(float("nan"))
        scal.fill_(float("nan"))
        torch.cuda.synchronize()
        st = prob.run_fixed_source_noalloc(opts, mesh.data_ptr(), 0, scal.data_ptr())
        got_mesh = mesh.cpu().numpy()
        got_scal = scal.cpu().numpy()
        assert np.all(np.isfinite(got_mesh)) and np.all(np.isfinite(got_scal)), f"call {k}"
        assert_tally_close(got_mesh, ref_mesh, f"mesh (call {k})")
        assert_tally_close(got_scal, ref_scal, f"scalars (call {k})")
        _same_bits(got_mesh, ref_mesh, f"mesh bits (call {k})")
        assert np.array_equal(st["final_by_type"], ref["final_by_type"]), f"call {k}"
        assert np.array_equal(st["events_by_type"], ref["events_by_type"]), f"call {k}"
        if k == 1:
            assert st["spills"] > 0 and st["refills"] > 0

    # requests beyond the static arena are refused before any device work
    with pytest.raises(tb.TransportError) as e:
        prob.run_fixed_source_noalloc(tb.RunOpts(n_histories=10, scheme=tb.SCHEME_ASYNC,
                                                 queue_capacity=MAX_QUEUE + 32),
                                      mesh.data_ptr(), 0, scal.data_ptr())
    assert e.value.status == tb.TR_ERR_INVALID
    prob.close()


@pytest.mark.parametrize("remap", [2, 512])
def test_noalloc_monolithic_samples_sources_in_the_loop(remap):
    """The allocation-free run has no pre-sampling buffer, so its monolithic
    kernel samples sources inside the loop (with deferred collisions at 512
    events per remap, whole events at 2): same results as the allocating run,
    which pre-samples them."""
    import torch
    from paper_2506_00263_gb300 import build
    build.build()
    prob = tb.Problem(inputs.c5g7_lattice())
    n = 50_021
    kw = dict(n_histories=n, seed=5, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO, remap_every=remap)
    ref = prob.run_fixed_source(tb.RunOpts(**kw))
    ref_mesh = prob.tally(tb.TALLY_MESH)
    ref_scal = prob.tally(tb.TALLY_SCALARS)
    mesh = torch.empty(ref_mesh.size, dtype=torch.float64, device="cuda")
    scal = torch.empty(3, dtype=torch.float64, device="cuda")
    st = prob.run_fixed_source_noalloc(tb.RunOpts(**kw), mesh.data_ptr(), 0, scal.data_ptr())
    assert np.array_equal(st["final_by_type"], ref["final_by_type"])
    assert np.array_equal(st["events_by_type"], ref["events_by_type"])
    assert_tally_close(mesh.cpu().numpy(), ref_mesh, "mesh")
    assert_tally_close(scal.cpu().numpy(), ref_scal, "scalars")
    _same_bits(mesh.cpu().numpy(), ref_mesh, "mesh bits")
    prob.close()


def test_noalloc_takes_no_device_memory_after_its_first_call():
    """After one call with given options (which may load that kernel), a
    further call leaves the device's free memory unchanged."""
    import torch
    from paper_2506_00263_gb300 import build
    build.build()
    prob = tb.Problem(inputs.c5g7_lattice())
    mesh = torch.empty(prob.tally_size(tb.TALLY_MESH), dtype=torch.float64, device="cuda")
    scal = torch.empty(3, dtype=torch.float64, device="cuda")
    opts = tb.RunOpts(n_histories=20_011, seed=9, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO,
                      remap_every=64)
    prob.run_fixed_source_noalloc(opts, mesh.data_ptr(), 0, scal.data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    first = mesh.cpu().numpy().copy()
    prob.run_fixed_source_noalloc(opts, mesh.data_ptr(), 0, scal.data_ptr())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    _same_bits(mesh.cpu().numpy(), first, "second call")
    prob.close()


def test_noalloc_continuous_energy_and_bin_limit():
    """A continuous-energy problem through the allocation-free run equals the
    allocating run; a problem with more tally bins than the static array
    holds is refused before any device work."""
    import torch
    from paper_2506_00263_gb300 import build
    build.build()
    prob = tb.Problem(inputs.ce_pin_cell(n_points=20000, n_res=60, n_ebins=100))
    kw = dict(n_histories=3_001, seed=2, scheme=tb.SCHEME_ASYNC, decomposition=tb.DECOMP_MONO, remap_every=64)
    ref = prob.run_fixed_source(tb.RunOpts(**kw))
    ref_e = prob.tally(tb.TALLY_ENERGY)
    ref_s = prob.tally(tb.TALLY_SCALARS)
    energy = torch.empty(ref_e.size, dtype=torch.float64, device="cuda")
    scal = torch.empty(3, dtype=torch.float64, device="cuda")
    st = prob.run_fixed_source_noalloc(tb.RunOpts(**kw), 0, energy.data_ptr(), scal.data_ptr())
    assert np.array_equal(st["events_by_type"], ref["events_by_type"])
    _same_bits(energy.cpu().numpy(), ref_e, "CE energy bits")
    assert_tally_close(scal.cpu().numpy(), ref_s, "CE scalars")
    prob.close()
    big = tb.Problem(inputs.cube_one_group(n_mesh=32))
    assert big.tally_size(tb.TALLY_MESH) + 3 > MAX_BINS
    mesh = torch.empty(big.tally_size(tb.TALLY_MESH), dtype=torch.float64, device="cuda")
    with pytest.raises(tb.TransportError) as e:
        big.run_fixed_source_noalloc(tb.RunOpts(n_histories=10, scheme=tb.SCHEME_ASYNC), mesh.data_ptr(), 0,
                                     scal.data_ptr())
    assert e.value.status == tb.TR_ERR_INVALID
    big.close()
