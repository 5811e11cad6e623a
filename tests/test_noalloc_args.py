"""Host-side argument checks of the allocation-free entry point's binding.

cbfs_run_noalloc takes raw pointers: a tensor of the wrong type or size would
be read or written past its end on the device.  The binding rejects such
tensors with ValueError before the library is called, so these checks run
without a GPU.
"""
import pytest
import torch

from paper_2410_17226_gb300 import cbfs


def _args(n=10, d=2):
    return dict(off=torch.zeros(n + 1, dtype=torch.int64), adj=torch.zeros(4, dtype=torch.int32),
                d=d, dist=torch.zeros(n, dtype=torch.uint8), masks=torch.zeros((d, n), dtype=torch.int64))


@pytest.mark.parametrize("field,value,words", [
    ("off", torch.zeros(11, dtype=torch.int32), "off must be torch.int64"),
    ("adj", torch.zeros(4, dtype=torch.int64), "adj must be torch.int32"),
    ("dist", torch.zeros(10, dtype=torch.int8), "dist must be torch.uint8"),
    ("masks", torch.zeros((2, 10), dtype=torch.int32), "masks must be torch.int64"),
    ("dist", torch.zeros(9, dtype=torch.uint8), "dist has 9 entries"),
    ("masks", torch.zeros((2, 9), dtype=torch.int64), "masks has shape"),
    ("masks", torch.zeros((1, 10), dtype=torch.int64), "masks has shape"),
    ("off", torch.zeros(1, dtype=torch.int64), "off must be 1-D"),
    ("adj", torch.zeros((2, 2), dtype=torch.int32), "adj must be 1-D"),
    ("off", [0] * 11, "off must be a torch.Tensor"),
])
def test_rejects_wrong_tensors(field, value, words):
    a = _args()
    a[field] = value
    with pytest.raises(ValueError, match=words):
        cbfs.run_noalloc(a["off"], a["adj"], [0], a["d"], a["dist"], a["masks"])


def test_rejects_host_tensors():
    a = _args()
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        cbfs.run_noalloc(a["off"], a["adj"], [0], a["d"], a["dist"], a["masks"])


def test_masks_ignored_when_d_is_zero():
    a = _args(d=0)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        cbfs.run_noalloc(a["off"], a["adj"], [0], 0, a["dist"], None)
