"""Write every preset as a JSON workload config into workloads/configs/
(``python -m workloads``).  The files can be edited and passed to
``workloads.preset`` / ``workloads.make_events`` or ``bench.py --workload``."""
import os

import workloads as W


def main() -> None:
    os.makedirs(W.CONFIG_DIR, exist_ok=True)
    for name in sorted(W.PRESETS):
        path = os.path.join(W.CONFIG_DIR, name + ".json")
        W.save_config(name, path)
        print(path)


if __name__ == "__main__":
    main()
