"""fempic_sort_noalloc: the sort entry point for callers that must not
allocate device memory while running (their device memory belongs to a
pool handed out up front, or they cannot absorb the synchronization a
cudaFree implies).  It must give the same result as fempic_sort, call after
call, while its scratch lives in a fixed area inside the library.

The order of particles inside one tet is unspecified for both entry points
(atomic slot claims), so the comparison is: the sorted tet ids position by
position, and, inside each tet, the same particles (matched by the original
index each particle carries in n_cross) with bit-identical state.
"""
import numpy as np
import pytest

from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _loaded():
    from paper_2208_12795_gb300 import build, capi
    build.build()
    capi.load()
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    return capi, FempicEnv, ParticleState


def _state(ParticleState, env, parts, prec, rng):
    st = ParticleState.from_host(parts, prec)
    env.locate(st)
    tet = st.tet.cpu().numpy()
    tet[rng.random(parts.n) < 0.01] = -1          # some unlocated particles (sorted last)
    st.tet.copy_(torch.from_numpy(tet).cuda())
    st.n_cross.copy_(torch.arange(parts.n, dtype=torch.int32, device="cuda"))   # original index
    return st


def _canonical(st):
    d = st.to_numpy()
    order = np.lexsort((d["n_cross"], np.where(d["tet"] >= 0, d["tet"], 1 << 30)))
    return d, {k: v[order] for k, v in d.items()}


def _check_same(ref, new, parts):
    dr, cr = _canonical(ref)
    dn, cn = _canonical(new)
    assert np.array_equal(dr["tet"], dn["tet"])              # the sorted key sequence is unique
    for k in cr:
        assert np.array_equal(cr[k], cn[k]), k             # same particles, same state, per tet
    sb = parts.species_begin
    for s in range(len(sb) - 1):                           # species ranges stay in place
        seg = dn["n_cross"][sb[s]:sb[s + 1]]
        assert np.all((seg >= sb[s]) & (seg < sb[s + 1]))


def test_sort_noalloc_matches_sort_two_calls_in_a_row():
    capi, FempicEnv, ParticleState = _loaded()
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        (I.kuhn_cube_mesh(8), 0, I.concat_species([I.uniform_maxwellian(40000, 1.0, rng),
                                                   I.uniform_maxwellian(23457, 2.0, rng, q=I.E_CHARGE,
                                                                        m=1836 * I.M_ELECTRON)])),
        (I.kuhn_cube_mesh(11, jitter=0.2, rng=rng), 1, I.uniform_maxwellian(70001, 5.0, rng)),
    ]
    for mesh, prec, parts in cases:                        # two calls in a row, different shapes
        env = FempicEnv.from_mesh(mesh, precision=prec)
        st = _state(ParticleState, env, parts, prec, rng)
        ref, new = st.empty_like(), st.empty_like()
        capi.fempic_sort(env.h, st.cstruct(), ref.cstruct(), stream)
        capi.fempic_sort_noalloc(env.h, st.cstruct(), new.cstruct(), stream)
        torch.cuda.synchronize()
        _check_same(ref, new, parts)
        env.close()


def test_sort_noalloc_rejects_more_keys_than_its_scratch():
    capi, FempicEnv, ParticleState = _loaded()
    mesh = I.kuhn_cube_mesh(37)                            # 303,918 tets
    env = FempicEnv.from_mesh(mesh)
    rng = np.random.default_rng(5)
    parts = I.concat_species([I.uniform_maxwellian(10, 1.0, rng) for _ in range(8)])
    assert 8 * (env.n_tets + 1) > capi.FEMPIC_SORT_NOALLOC_MAX_KEYS
    st = ParticleState.from_host(parts, 0)
    env.locate(st)
    out = st.empty_like()
    lib = capi.load()
    import ctypes as C
    rc = lib.fempic_sort_noalloc(env.h, C.byref(st.cstruct()), C.byref(out.cstruct()),
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == capi.FEMPIC_EINVAL
    assert "exceeds the fixed scratch" in capi.fempic_last_error()
    env.close()


def test_sort_noalloc_takes_no_device_memory_after_the_first_call():
    """After a warm-up call (which looks up the scratch area's address and
    loads the kernels), further calls, on a larger key count than before,
    leave the device's free memory exactly unchanged."""
    capi, FempicEnv, ParticleState = _loaded()
    rng = np.random.default_rng(99)
    stream = torch.cuda.current_stream().cuda_stream
    small = FempicEnv.from_mesh(I.kuhn_cube_mesh(5), precision=1)
    big = FempicEnv.from_mesh(I.kuhn_cube_mesh(40), precision=1)        # 384,000 tets
    ps = I.uniform_maxwellian(5000, 1.0, rng)
    pb = I.concat_species([I.uniform_maxwellian(300_000, 1.0, rng),
                           I.uniform_maxwellian(200_000, 2.0, rng, q=I.E_CHARGE, m=1836 * I.M_ELECTRON)])
    ss, sb = _state(ParticleState, small, ps, 1, rng), _state(ParticleState, big, pb, 1, rng)
    outs, outb = ss.empty_like(), sb.empty_like()
    capi.fempic_sort_noalloc(small.h, ss.cstruct(), outs.cstruct(), stream)     # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        capi.fempic_sort_noalloc(big.h, sb.cstruct(), outb.cstruct(), stream)
        capi.fempic_sort_noalloc(small.h, ss.cstruct(), outs.cstruct(), stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert 2 * (big.n_tets + 1) > 100 * (small.n_tets + 1)              # far more keys than the warm-up
    ref = sb.empty_like()
    capi.fempic_sort(big.h, sb.cstruct(), ref.cstruct(), stream)
    torch.cuda.synchronize()
    _check_same(ref, outb, pb)
    big.close()
    small.close()
