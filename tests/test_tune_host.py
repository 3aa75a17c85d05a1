"""CPU checks of the batch autotuner's host logic: the batch signature that
keys its cache (order-free, N bucketed to the next power of two, kind and
width kept apart)."""
from paper_2111_05778_gb300 import tune


class _Mlp:
    def __init__(self, width):
        self.width = width


class _Csg:
    pass


def test_signature_ignores_order_and_buckets_n():
    a = tune.signature([_Mlp(64), _Csg(), _Mlp(256)], [128, 1000, 384], "bf16")
    b = tune.signature([_Mlp(256), _Mlp(64), _Csg()], [500, 100, 1024], "bf16")
    assert a == b == "bf16:csg@1024,mlp256@512,mlp64@128"
    assert tune.signature([_Csg()], [129], "fp32") == "fp32:csg@256"
    assert tune.signature([_Mlp(64)], [64], "fp32") != tune.signature([_Mlp(128)], [64], "fp32")

