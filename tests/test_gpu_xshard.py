"""The x-column split of one stack across GPUs, run here as separate calls
on one GPU: each part is the live view of a column range with its own plan
(same output grid), and the concatenation of the parts is the whole stack's
live view bit for bit, for the periodic, fast and general kernels."""
import pytest

import opm_synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape,parts", [
    ((200, 64, 512, 35.0, 0.3, 0.1), 4),      # periodic kernel
    ((40, 70, 264, 35.0, 0.3, 0.1), 3),       # ragged x tile
    ((64, 128, 128, 30.0, 0.4, 0.115), 3),    # fast kernel
    ((16, 20, 64, 35.0, 0.05, 0.1), 2),       # general kernel (pixel > step)
    ((33, 50, 203, 45.0, 0.2, 0.115), 4),     # odd width: the last part is ragged
])
def test_xshard_parts_concatenate_to_the_whole(lib, shape, parts):
    from paper_2211_00645_gb300 import dist as pdist
    R = opm_synth.raw_stack(opm_synth.StackConfig("x", *shape, n_blobs=12, sigma=(1.0, 3.0),
                                                  amp=(200.0, 4000.0), seed=17))
    raw = to_dev(R, torch)
    whole = lib.project(lib.Plan(*shape), raw, zmip=True, ymip=True)
    zs, ys = [], []
    for r in range(parts):
        x0, x1 = pdist.xshard(shape[2], r, parts)
        z, y = pdist.project_xshard(shape[3:], raw[:, :, x0:x1].contiguous())
        zs.append(z)
        ys.append(y)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(zs, dim=1), whole["zmip"])
    assert torch.equal(torch.cat(ys, dim=1), whole["ymip"])
