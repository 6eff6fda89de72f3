"""The input generators: the torch evaluation of the tube density reproduces
the numpy one (same seeded draws, same Gaussians and images)."""
import numpy as np
import pytest

from paper_0812_0244_gb300 import synthetic as S


@pytest.mark.parametrize("shape,shift,rot", [((24, 36, 36), 0.3, 7.0), ((16, 30, 40), 2.0, 33.0)])
def test_tube_density_torch_matches_numpy(shape, shift, rot):
    pytest.importorskip("torch")
    d = S.tube_density(5, shape=shape, shift_ang=shift, rot_deg=rot)
    n, L, na = S.tube_density_torch(5, shape=shape, shift_ang=shift, rot_deg=rot, device="cpu")
    assert na == d["natoms"] == 240
    np.testing.assert_allclose(L, d["L"])
    np.testing.assert_allclose(n.numpy(), d["n"], rtol=1e-12, atol=1e-15)


def test_tube_charge_is_four_electrons_per_site():
    d = S.tube_density(1, shape=(48, 96, 96))
    dOmega = np.prod(d["L"]) / d["n"].size
    floor = 1e-6 * np.prod(d["L"])
    assert abs((d["n"].sum() * dOmega - floor) / (4.0 * d["natoms"]) - 1.0) < 1e-3


def test_alike_sites_have_the_outer_walls_screw_symmetry():
    """With one set of Gaussian parameters per wall the outer (10,10) wall
    is unchanged by its screw operation (half the axial period with 18
    degrees) and by a full period; independent parameters per site are not."""
    shape = (24, 48, 48)
    ref = S.tube_density(7, shape=shape, sites_alike=True)["n"]
    for z, phi in ((0.5 * S.T_ARM, 18.0), (S.T_ARM, 0.0), (0.0, 36.0)):
        d = S.tube_density(7, shape=shape, shift_ang=z, rot_deg=phi, sites_alike=True)["n"]
        assert np.abs(d - ref).max() <= 1e-12 * ref.max()
    d = S.tube_density(7, shape=shape, shift_ang=0.5 * S.T_ARM, rot_deg=18.0)["n"]
    assert np.abs(d - S.tube_density(7, shape=shape)["n"]).max() > 1e-3 * ref.max()
