"""Slab decomposition along z on one GPU: the lattice split into slabs with one halo
plane per face, halo populations packed, copied between the slab handles and
unpacked after every pull step (olb_set_active_planes, olb_halo_pack,
olb_halo_unpack).  The interior of every slab must equal the single lattice bit
for bit after every step count, with walls crossing the cuts, a moving lid, a
porous forced flow, a periodic z axis whose cut wraps around, and every storage
type; the statistics summed over the slabs' active planes equal the single
lattice's."""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import cavity_case, porous_channel_case, tgv3d_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11752_gb300 import build, olb as _olb
    build.build()
    _olb.load()
    return _olb


def _with_halo(field, z0, z1, periodic_z, fill):
    """Planes z0 .. z1 of a [..., nz, ny, nx] field plus one plane on each side:
    the neighbouring planes, wrapped on a periodic z axis, else `fill`."""
    nz = field.shape[-3]
    planes = []
    for z in range(z0 - 1, z1 + 2):
        if 0 <= z < nz or periodic_z:
            planes.append(field[..., z % nz, :, :])
        else:
            planes.append(np.full_like(field[..., 0, :, :], fill))
    return np.ascontiguousarray(np.stack(planes, axis=-3))


def _lattice(olb, case, material, periodic, dtype, gamma):
    import torch

    nz, ny, nx = material.shape
    lat = olb.Lattice(case.d, (nx, ny, nz), dtype=dtype, scheme="pull")
    lat.set_material(torch.from_numpy(material.reshape(-1).copy()).cuda(), periodic)
    for k, v in case.walls.items():
        lat.set_wall_velocity(k, v)
    lat.set_bgk(case.tau)
    lat.set_force(case.force)
    if gamma is not None:
        lat.set_porosity(torch.from_numpy(np.ascontiguousarray(gamma).reshape(-1)).cuda())
    return lat


def _run(olb, case, dtype, cuts, checks):
    import torch

    m = case.material
    periodic_z = bool(case.periodic & 4)
    single = _lattice(olb, case, m, case.periodic, dtype, case.gamma)
    f0 = case.gpu(dtype, "pull").get_populations().cpu().numpy()  # the case's initial state
    single.set_populations(torch.from_numpy(f0).cuda())
    slabs = []
    for z0, z1 in cuts:
        ms = _with_halo(m, z0, z1, periodic_z, I.VOID if hasattr(I, "VOID") else 0)
        gs = None if case.gamma is None else _with_halo(case.gamma, z0, z1, periodic_z, 1.0)
        s = _lattice(olb, case, ms, case.periodic & 3, dtype, gs)
        s.set_populations(torch.from_numpy(_with_halo(f0, z0, z1, periodic_z, 0.0)).cuda())
        s.set_active_planes(1, z1 - z0 + 1)
        slabs.append(s)
    up = [s.halo_buffer() for s in slabs]    # packed at the high face, for the slab above
    down = [s.halo_buffer() for s in slabs]  # packed at the low face, for the slab below
    P = len(slabs)
    done = 0
    for target in checks:
        while done < target:
            single.step(1)
            for s in slabs:
                s.step(1)
            for k, s in enumerate(slabs):
                s.halo_pack(1, up[k])
                s.halo_pack(0, down[k])
            for k, s in enumerate(slabs):
                if k > 0 or periodic_z:
                    s.halo_unpack(0, up[(k - 1) % P])
                if k < P - 1 or periodic_z:
                    s.halo_unpack(1, down[(k + 1) % P])
            done += 1
        fs = single.get_populations().cpu().numpy()
        for (z0, z1), s in zip(cuts, slabs):
            got = s.get_populations().cpu().numpy()[:, 1:-1]
            assert np.array_equal(got, fs[:, z0:z1 + 1]), (target, z0, z1)
    stats = single.diagnostics()
    parts = np.array([s.diagnostics() for s in slabs])
    assert abs(parts[:, 0].sum() - stats[0]) <= 1e-12 * stats[0]
    assert abs(parts[:, 4].sum() - stats[4]) <= 1e-9 * stats[4]
    assert parts[:, 5].max() == stats[5]
    for s in slabs + [single]:
        s.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16", "bf16"])
def test_slabs_of_a_lid_driven_cavity(olb, dtype):
    case = cavity_case(26, 20, 18)
    _run(olb, case, dtype, [(0, 8), (9, 17)], [1, 2, 7, 25])


def test_slabs_of_a_forced_porous_channel_with_a_moving_wall(olb):
    case = porous_channel_case(nx=24, ny=12, nz=16, moving=True)
    _run(olb, case, "f32", [(0, 4), (5, 10), (11, 15)], [3, 20])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_slabs_of_a_periodic_vortex_wrap_around(olb, dtype):
    case = tgv3d_case(n=18)
    _run(olb, case, dtype, [(0, 5), (6, 11), (12, 17)], [1, 4, 30])


def test_halo_calls_check_their_state(olb):
    import torch

    case = cavity_case(12, 10, 8)
    g = case.gpu("f32", "pull")
    buf = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(olb.OlbError) as e:
        g.halo_pack(1, buf)  # no halo planes set
    assert e.value.status == -4
    g.set_active_planes(1, 6)
    with pytest.raises(olb.OlbError) as e:
        g.halo_pack(1, buf)  # state before any step
    assert e.value.status == -4
    g.step(1)
    g.halo_pack(1, buf)
    with pytest.raises(olb.OlbError):
        g.halo_pack(2, buf)
    with pytest.raises(olb.OlbError):
        g.set_active_planes(3, 2)
    g.set_active_planes(-1, -1)
    g.close()
