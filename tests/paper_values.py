"""Numbers printed in the paper, read from tests/golden/paper_values.txt (each line:
key, value, citation).  Module constants, so that a missing key fails at import."""
from pathlib import Path

GOLDEN = Path(__file__).parent / "golden" / "paper_values.txt"


def load(path: Path = GOLDEN) -> dict[str, tuple[float, str]]:
    """{key: (value, citation)} for every non-comment line of the fixture."""
    out = {}
    for line in path.read_text().splitlines():
        if not line.strip() or line.lstrip().startswith("#"):
            continue
        key, value, cite = line.split(None, 2)
        assert key not in out, f"duplicate key {key}"
        out[key] = (float(value), cite.strip())
    return out


PRINTED = {k: v for k, (v, _) in load().items()}
NUGGET_EPSILON_FP64 = PRINTED["nugget_epsilon_fp64"]
STENCIL_PIXELS = {1: int(PRINTED["stencil_pixels_y1"]), 2: int(PRINTED["stencil_pixels_y2"])}
LENSED_L2_NSIDE4096 = PRINTED["lensed_l2_nside4096_lmax4096"]
SUPERSAMPLE_2048_4096_9NGB = PRINTED["supersample_2048_4096_9ngb"]
