"""Argument checks of the bt_pair_dense_energy_noalloc binding, on the CPU.

The C entry point receives bare device pointers and cannot tell a float64
depth map, a short buffer or a tensor of another GPU from a correct one; the
binding must reject each of these before the call.  Stand-in tensors carry
the attributes the check reads (no GPU needed)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2108_00516_gb300.bt import noalloc_argument_error  # noqa: E402

W, H = 16, 12


class Fake:
    def __init__(self, dtype, numel, device=0, cuda=True, contiguous=True):
        self.dtype, self._n, self.is_cuda, self._c = dtype, numel, cuda, contiguous
        self.device = torch.device("cuda", device) if cuda else torch.device("cpu")

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def good():
    return dict(depth_a=Fake(torch.float32, W * H), normals_a=Fake(torch.float32, 3 * W * H),
                mask_a=Fake(torch.uint8, W * H), depth_b=Fake(torch.float32, W * H),
                normals_b=Fake(torch.float32, 3 * W * H), mask_b=Fake(torch.bool, W * H),
                out=Fake(torch.float64, 2))


def err(**over):
    a = good()
    a.update(over)
    return noalloc_argument_error(torch, 0, (W, H), (W, H), **a)


def test_accepts_correct_buffers():
    assert err() == ""


@pytest.mark.parametrize("over,words", [
    (dict(depth_a=Fake(torch.float64, W * H)), "depth_a must be float32"),
    (dict(depth_b=Fake(torch.float32, W * H - 1)), "depth_b must be float32 with W*H"),
    (dict(normals_a=Fake(torch.float32, W * H)), "normals_a must be float32 with 3*W*H"),
    (dict(normals_b=Fake(torch.float16, 3 * W * H)), "normals_b must be float32"),
    (dict(mask_a=Fake(torch.int32, W * H)), "mask_a must be uint8 or bool"),
    (dict(mask_b=Fake(torch.uint8, W * H + 5)), "mask_b must be uint8 or bool with W*H"),
    (dict(out=Fake(torch.float32, 2)), "out must be float64"),
    (dict(out=Fake(torch.float64, 1)), "at least 2"),
    (dict(depth_a=Fake(torch.float32, W * H, cuda=False)), "contiguous CUDA tensor"),
    (dict(normals_b=Fake(torch.float32, 3 * W * H, contiguous=False)), "contiguous CUDA tensor"),
    (dict(mask_a=Fake(torch.uint8, W * H, device=1)), "not cuda:0"),
])
def test_rejects(over, words):
    assert words in err(**over)
