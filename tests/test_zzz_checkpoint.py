"""Key and ciphertext checkpoints through the library: keys saved to a file,
erased and loaded back equal the oracle's keys bit for bit and rotate to the
same bits; loading over resident keys overwrites them in place; a residue at
its modulus is refused before any copy and leaves the key as it was; a
ciphertext saved and loaded keeps its limbs, level and scale."""
import pytest

import gpu_common
from paper_2510_03996_gb300 import checkpoint as CK
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu


def test_key_and_ciphertext_checkpoint(tmp_path):
    pr = gpu_common.Pair("small_n12", rot_steps=[1, 5])
    g = pr.g
    g.relinkeygen(pr.sk)
    g1, g5 = g.galois_elt(1), g.galois_elt(5)
    assert g.key_list() == sorted([0, g1, g5])
    m = synth.small_int_poly(21, 0, pr.N, 1 << 40)
    ct, _ = pr.encrypt_both(m, nonce=21)
    before = g.ct_download(g.rotate(ct, 5))

    path = str(tmp_path / "keys.ck")
    assert CK.save_keys(g, path) == sorted([0, g1, g5])
    g.key_erase(g5)
    assert g5 not in g.key_list()
    assert CK.load_keys(g, path, [g5]) == [g5]
    assert gpu_common.mismatch(g.key_download(g5), pr.okeys[g5]) == 0
    assert gpu_common.mismatch(g.ct_download(g.rotate(ct, 5)), before) == 0

    # over resident keys: overwritten in place with the same values
    assert CK.load_keys(g, path) == sorted([0, g1, g5])
    assert gpu_common.mismatch(g.key_download(g1), pr.okeys[g1]) == 0
    assert gpu_common.mismatch(g.ct_download(g.rotate(ct, 5)), before) == 0

    bad = g.key_download(g1)
    bad[0, 0, 0, 3] = g.moduli[0]
    with pytest.raises(pr.F.FheonError) as e:
        g.key_upload(g1, bad)
    assert e.value.code == -1
    assert gpu_common.mismatch(g.key_download(g1), pr.okeys[g1]) == 0

    cpath = str(tmp_path / "ct.ck")
    c3 = g.drop_level(ct, 3)
    CK.save_ct(g, c3, cpath)
    back = CK.load_ct(g, cpath)
    assert g.ct_info(back) == g.ct_info(c3)
    assert gpu_common.mismatch(g.ct_download(back), g.ct_download(c3)) == 0
